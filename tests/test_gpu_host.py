"""tdm_solve_host: right-hand sides and solutions in host memory, copied in
chunks that overlap the solves; the result equals the device solve bit for
bit (every column is solved by the same tile arithmetic)."""
import numpy as np
import pytest
import torch

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("precision", ["fp32_refined", "fp32", "fp64"])
@pytest.mark.parametrize("N,chunk", [(37, 0), (1000, 0), (1000, 96), (3000, 512)])
@pytest.mark.parametrize("pinned", [True, False])
def test_equals_the_device_solve(precision, N, chunk, pinned):
    import paper_0901_2859_gb300 as tdm
    from paper_0901_2859_gb300 import workloads
    s = workloads.plain_fp64(seed=N, n=1500, N=N)
    plan = tdm.prepare(s.a, s.b, device="cuda:0")
    dt = torch.float64 if precision == "fp64" else torch.float32
    F = torch.from_numpy(s.F).to(dt)
    if pinned:
        F = F.pin_memory()
    X = plan.solve_host(F, precision, chunk=chunk)
    torch.cuda.synchronize()
    ref = plan.solve(F.cuda(), precision).cpu()
    assert torch.equal(X, ref)
    plan.close()


def test_strided_host_arrays_and_repeated_calls():
    import paper_0901_2859_gb300 as tdm
    from paper_0901_2859_gb300 import workloads
    s = workloads.plain_fp64(seed=1, n=700, N=300)
    plan = tdm.prepare(s.a, s.b, device="cuda:0")
    big = torch.zeros((700, 512), dtype=torch.float32).pin_memory()
    big[:, :300] = torch.from_numpy(s.F).float()
    out = torch.zeros((700, 400), dtype=torch.float64).pin_memory()
    for _ in range(3):   # the staging buffers are reused across calls
        plan.solve_host(big[:, :300], "fp32_refined", out=out[:, :300], chunk=64)
    torch.cuda.synchronize()
    assert torch.equal(out[:, :300], plan.solve(big[:, :300].cuda(), "fp32_refined").cpu())
    assert torch.count_nonzero(out[:, 300:]) == 0
    with pytest.raises(TypeError):
        plan.solve_host(big.cuda(), "fp32")
    plan.close()
