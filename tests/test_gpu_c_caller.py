"""A plain C program calling libpat (pat_plan_create, pat_forward, pat_adjoint_grad, pat_status)
gives the traces, J and gradients of the Python binding on the same inputs: the two callers reach
the same kernels, so they agree to FP32 rounding (1e-6 relative)."""
import os
import subprocess

import numpy as np
import pytest

import pat_synth as ps

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def test_c_caller_matches_python_binding(tmp_path):
    from tests._problems import grid_params, gpu_plan, rel_l2, small_case
    from tests.c.build_c_caller import build_c_caller
    exe = str(tmp_path / "pat_c_caller")
    build_c_caller(exe)
    K, nt, M = 3, 150, 20
    c, p0, xy = small_case(n=40, K=K, M=M, nt=nt, seed=11)
    gp = grid_params(40, nt)
    plan = gpu_plan(gp, xy, K, ckpt_every=16)
    dev = lambda a: torch.as_tensor(np.ascontiguousarray(a), dtype=torch.float32, device="cuda")
    y = plan.forward(dev(c), dev(p0)).cpu().numpy()
    ym = ps.add_noise(y, ps.rng_for(211)).astype(np.float32)
    w = ps.noise_weights(ym).astype(np.float32)
    J, gp0, gc = plan.adjoint_grad(dev(c), dev(0.5 * p0), dev(ym), dev(w))
    d = str(tmp_path)
    with open(os.path.join(d, "meta.txt"), "w") as f:
        f.write(f"{gp['n']} {gp['pml']} {gp['dx']!r} {gp['dt']!r} {gp['nt']} {gp['c_ref']!r} {gp['rho0']!r} "
                f"{gp['pml_alpha']!r} {gp['c_bg']!r} {M} {K} 16\n")
    np.ascontiguousarray(c, dtype=np.float32).tofile(os.path.join(d, "c.f32"))
    np.ascontiguousarray(0.5 * p0, dtype=np.float32).tofile(os.path.join(d, "p0.f32"))
    ym.tofile(os.path.join(d, "y_meas.f32"))
    w.tofile(os.path.join(d, "w.f32"))
    np.ascontiguousarray(xy, dtype=np.float64).tofile(os.path.join(d, "xy.f64"))
    r = subprocess.run([exe, d], capture_output=True, text=True, timeout=300)
    assert r.returncode == 0, r.stdout + r.stderr
    assert r.stdout.split()[3] == "0"   # pat_status: no flag
    y_c = np.fromfile(os.path.join(d, "y.f32"), dtype=np.float32).reshape(K, nt, M)
    gp0_c = np.fromfile(os.path.join(d, "grad_p0.f32"), dtype=np.float32).reshape(K, 40, 40)
    gc_c = np.fromfile(os.path.join(d, "grad_c.f32"), dtype=np.float32).reshape(40, 40)
    J_c = float(np.fromfile(os.path.join(d, "J.f64"), dtype=np.float64)[0])
    # the C caller's traces are those of p0 / 2 (its forward runs on the gradient's inputs)
    y_half = plan.forward(dev(c), dev(0.5 * p0)).cpu().numpy()
    assert rel_l2(y_c, y_half) <= 1e-6
    assert abs(J_c - float(J)) <= 1e-6 * abs(float(J))
    assert rel_l2(gp0_c, gp0.cpu().numpy()) <= 1e-6
    assert rel_l2(gc_c, gc.cpu().numpy()) <= 1e-6
