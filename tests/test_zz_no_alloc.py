"""The allocation-free momentum/energy reduction (sfmm_reduce_noalloc).

Some callers cannot call cudaMalloc -- code that draws every byte of device
memory from its own reserved pool, or that must keep the device's memory
footprint fixed while it runs -- so the library offers one entry point whose
scratch is a fixed array inside the library.  This test calls it through the
C ABI on the outputs of a gravity solve, twice in a row (the second call
reuses the array the first one left behind), and checks both results against
the sums the ordinary gravity entry point reports, within the FP64 tolerance
the other parity tests use.  It lives in a file of its own that pytest
collects last, and runs the same alone or after the other tests.
"""
import numpy as np
import pytest

import workloads
from gpu_helpers import TOL_FP64

pytestmark = pytest.mark.gpu


def test_noalloc_reduction_matches_gravity_stats_twice():
    import torch

    from paper_2602_05804_gb300 import sfmm

    pos, m, h = workloads.plummer(50_000, 123)
    s = sfmm.Solver(0, "fp64")
    s.build(pos, m, h, 16)
    acc, pot = s.gravity(0.5, 2)
    st = s.stats()
    ref = np.array(st["momentum"] + [st["abs_momentum"], st["W"]])
    mass = torch.from_numpy(m).cuda()
    out = torch.full((5,), float("nan"), dtype=torch.float64, device="cuda")
    scale = np.array([st["abs_momentum"]] * 4 + [abs(st["W"])])
    # the first call in a context looks up the array (and the driver may load
    # the library's module holding it); the calls after it allocate nothing
    sfmm.sfmm_reduce_noalloc(len(m), mass, acc, pot, out, torch.cuda.current_stream().cuda_stream)
    torch.cuda.synchronize()
    got_calls = []
    for call in range(2):
        out.fill_(float("nan"))
        torch.cuda.synchronize()
        # nothing may be allocated by the call itself: neither device memory
        # as the driver sees it nor torch's allocator changes across it
        free0, allocated0 = torch.cuda.mem_get_info()[0], torch.cuda.memory_allocated()
        sfmm.sfmm_reduce_noalloc(len(m), mass, acc, pot, out, torch.cuda.current_stream().cuda_stream)
        torch.cuda.synchronize()
        assert torch.cuda.mem_get_info()[0] == free0, call
        assert torch.cuda.memory_allocated() == allocated0, call
        got = out.cpu().numpy()
        got_calls.append(got)
        assert np.all(np.isfinite(got)), call
        assert np.all(np.abs(got - ref) <= TOL_FP64 * scale), (call, got, ref)
    np.testing.assert_array_equal(got_calls[0], got_calls[1])
    # a different, smaller input on the same scratch: matches its own sums
    acc2 = acc[:1000].contiguous()
    pot2 = pot[:1000].contiguous()
    sfmm.sfmm_reduce_noalloc(1000, mass[:1000].contiguous(), acc2, pot2, out, torch.cuda.current_stream().cuda_stream)
    torch.cuda.synchronize()
    a = acc2.cpu().numpy() * m[:1000, None]
    exp = np.concatenate([a.sum(0), [np.abs(a).sum(), 0.5 * (m[:1000] * pot2.cpu().numpy()).sum()]])
    np.testing.assert_allclose(out.cpu().numpy(), exp, rtol=1e-12, atol=1e-12 * np.abs(a).sum())


def test_noalloc_rejects_sizes_beyond_the_maximum():
    import torch

    from paper_2602_05804_gb300 import sfmm

    t = torch.zeros(16, dtype=torch.float64, device="cuda")
    for n in (0, sfmm.SFMM_NOALLOC_MAX_N + 1):
        with pytest.raises(sfmm.SFMMError) as e:
            sfmm.sfmm_reduce_noalloc(n, t, t, t, t)
        assert e.value.code == sfmm.SFMM_EINVAL
