"""Cases run by tests/test_gpu_debug_bounds.py with the release library and, in a child
process with PAT_DEBUG_BOUNDS=1, with the bounds-checked library: forward traces and
gradients of a generic-kernel grid with ragged tiles and checkpoint segments, and of the
300-point grid with the fixed-size passes (default and TMA-staged variants).

Run as a script (``python tests/_debug_bounds_cases.py out.npz``) it builds and loads the
bounds-checked library, checks its self-test and writes the results, the status words and
the library's build flag to out.npz.
"""
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
for p in (ROOT,):
    if p not in sys.path:
        sys.path.insert(0, p)


def run_cases():
    import torch
    import pat_synth as ps
    from tests._problems import grid_params, gpu_plan, small_case
    from paper_2505_08482_gb300 import _binding as B
    dev = torch.device("cuda", 0)
    f32 = lambda a: torch.as_tensor(np.ascontiguousarray(a), dtype=torch.float32, device=dev)
    out = {}
    rng = ps.rng_for(77)
    c, p0, xy = small_case(n=40, K=3, M=20, nt=150, seed=5)
    c2 = ps.ellipse_phantom(256, 4, rng)
    p02 = np.stack([ps.blob_p0(256, 4, rng) for _ in range(2)])
    xy2 = ps.circle_sensors(256, 64, 1e-4, phase=0.1)
    cases = [("generic40", grid_params(40, 150), c, p0, xy, None),
             ("fixed300_v5", grid_params(256, 40), c2, p02, xy2, 5),
             ("fixed300_v3", grid_params(256, 40), c2, p02, xy2, 3)]
    for name, gp, cc, pp, sx, variant in cases:
        plan = gpu_plan(gp, sx, pp.shape[0], ckpt_every=16)
        if variant is not None:
            plan.variant = variant
        y = plan.forward(f32(cc), f32(pp))
        st_f = plan.status(B.PAT_WS_FORWARD)
        ym = 0.9 * y + 0.01
        J, gp0, gc = plan.adjoint_grad(f32(cc), f32(0.5 * pp), ym, f32(np.ones(pp.shape[0])))
        st_g = plan.status(B.PAT_WS_GRADIENT)
        torch.cuda.synchronize()
        out[f"{name}_y"] = y.cpu().numpy()
        out[f"{name}_J"] = np.asarray(J.cpu().numpy(), dtype=np.float64)
        out[f"{name}_gp0"] = gp0.cpu().numpy()
        out[f"{name}_gc"] = gc.cpu().numpy()
        out[f"{name}_status"] = np.array([st_f, st_g])
    # self-test of the check: an index one past the end
    s = torch.zeros(1, dtype=torch.int32, device=dev)
    B.check(B.lib().pat_selftest_bounds(s.data_ptr(), torch.cuda.current_stream().cuda_stream),
            "pat_selftest_bounds")
    torch.cuda.synchronize()
    out["selftest_status"] = s.cpu().numpy()
    out["debug_bounds"] = np.array(B.lib().pat_debug_bounds())
    return out


if __name__ == "__main__":
    assert os.environ.get("PAT_DEBUG_BOUNDS") == "1", "run with PAT_DEBUG_BOUNDS=1"
    import paper_2505_08482_gb300 as pkg
    pkg.build(debug=True)
    np.savez(sys.argv[1], **run_cases())
