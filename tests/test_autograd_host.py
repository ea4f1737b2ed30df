"""Mechanics of the autograd wrapper on the CPU, with a stand-in plan.

The stand-in is a small linear map y = A(c) p0 whose forward stores a
"checkpoint" (its inputs' checksum) in the workspace it is given, and whose
vjp checks that it receives that same workspace, as pat_vjp needs the
checkpoints of the matching pat_forward.  This pins the wrapper's contract:
one workspace per forward, handed to the backward, kept for a second backward
when the graph is retained, and gradients routed to the right inputs.
"""
import pytest

torch = pytest.importorskip("torch")

from paper_2505_08482_gb300.autograd import pat_forward  # noqa: E402


class StandInPlan:
    device = "cpu"

    def __init__(self, K=2, n=3, nt=4, m=5, seed=0):
        g = torch.Generator().manual_seed(seed)
        self.M = torch.randn(nt * m, n * n, generator=g, dtype=torch.float32)
        self.shape = (K, nt, m)
        self.calls = []

    def workspace_bytes(self, kind):
        return 64

    def forward(self, c, p0, keep_checkpoints=False, ws=None):
        assert keep_checkpoints and ws is not None and ws.numel() == 64
        ws.view(torch.float32)[0] = float(p0.sum() + c.sum())          # the "checkpoint"
        self.calls.append(("forward", ws.data_ptr()))
        # y_k = M (c * p0_k): linear in p0, bilinear in (c, p0)
        return torch.stack([self.M @ (c * p).reshape(-1) for p in p0]).reshape(self.shape)

    def vjp(self, c, p0, ybar, ws=None):
        assert ws is not None and float(ws.view(torch.float32)[0]) == pytest.approx(float(p0.sum() + c.sum()))
        self.calls.append(("vjp", ws.data_ptr()))
        gq = torch.stack([(self.M.T @ yb.reshape(-1)).reshape(c.shape) for yb in ybar])
        return gq * c, (gq * p0).sum(0)


def test_gradients_match_autograd_of_the_same_map():
    plan = StandInPlan()
    p0 = torch.rand(2, 3, 3, requires_grad=True)
    c = (1500 + torch.rand(3, 3)).requires_grad_(True)
    y = pat_forward(p0, c, plan)
    (y * torch.linspace(-1, 1, y.numel()).reshape(y.shape)).sum().backward()
    p0r = p0.detach().clone().requires_grad_(True)
    cr = c.detach().clone().requires_grad_(True)
    yr = torch.stack([plan.M @ (cr * p).reshape(-1) for p in p0r]).reshape(y.shape)
    (yr * torch.linspace(-1, 1, y.numel()).reshape(y.shape)).sum().backward()
    torch.testing.assert_close(p0.grad, p0r.grad)
    torch.testing.assert_close(c.grad, cr.grad)
    assert [k for k, _ in plan.calls] == ["forward", "vjp"] and plan.calls[0][1] == plan.calls[1][1]


def test_retained_graph_backs_up_twice_with_the_same_checkpoints():
    plan = StandInPlan(seed=1)
    p0 = torch.rand(2, 3, 3, requires_grad=True)
    c = (1500 + torch.rand(3, 3)).requires_grad_(True)
    y = pat_forward(p0, c, plan)
    y.sum().backward(retain_graph=True)
    g1 = p0.grad.clone()
    y.sum().backward()
    torch.testing.assert_close(p0.grad, 2 * g1)
    ptrs = {p for _, p in plan.calls}
    assert [k for k, _ in plan.calls] == ["forward", "vjp", "vjp"] and len(ptrs) == 1


def test_two_forwards_keep_separate_workspaces():
    plan = StandInPlan(seed=2)
    p0 = torch.rand(2, 3, 3, requires_grad=True)
    c = (1500 + torch.rand(3, 3)).requires_grad_(True)
    ya = pat_forward(p0, c, plan)
    yb = pat_forward(2 * p0, c, plan)           # a second forward before either backward
    (ya.sum() + yb.sum()).backward()
    fw = [p for k, p in plan.calls if k == "forward"]
    vj = [p for k, p in plan.calls if k == "vjp"]
    assert len(set(fw)) == 2 and set(vj) == set(fw)
    assert c.grad is not None and p0.grad is not None


def test_only_requested_gradients_are_returned():
    plan = StandInPlan(seed=3)
    p0 = torch.rand(2, 3, 3, requires_grad=True)
    c = 1500 + torch.rand(3, 3)
    pat_forward(p0, c, plan).sum().backward()
    assert p0.grad is not None and c.grad is None


def test_iteration_log_is_one_json_object_per_line(tmp_path):
    import json
    from paper_2505_08482_gb300.solver import write_report_jsonl
    rows = [dict(level=0, it=0, J=2.0, gnorm=1.0, alpha=1.0, trials=1, J_new=1.5, ms=3.0, Ec=4.0, Ep0=50.0),
            dict(level=1, it=0, J=1.5, gnorm=0.5, alpha=0.5, trials=2, J_new=1.0, ms=2.5, Ec=2.0, Ep0=30.0)]
    p = tmp_path / "log.jsonl"
    write_report_jsonl(rows, p, instance=7)
    write_report_jsonl(rows[:1], p, instance=8)
    lines = [json.loads(l) for l in open(p)]
    assert [l["instance"] for l in lines] == [7, 7, 8]
    assert lines[1]["level"] == 1 and lines[1]["Ec"] == 2.0 and lines[0]["J_new"] == 1.5
