"""chisao_dedup_noalloc against the context-based deduplication.

The allocation-free entry point serves callers that cannot allocate device
memory (a host memory pool that has reserved the whole device, a plug-in handed
only its buffers, loops that must not synchronize on cudaMalloc/cudaFree).  It
must return exactly the
masks and counts of the context path (Phase 3 through chisao_run_phase), on two
calls in a row that share its one static scratch array.  This file is named so
that pytest collects it last.
"""
import ctypes as C

import numpy as np
import pytest

import gpu_util as U
from oracle import method as M
from paper_2606_26164_gb300 import chisao as CH
from paper_2606_26164_gb300 import inputs as I

pytestmark = pytest.mark.gpu


def _case(seed, N, d):
    rng = np.random.default_rng(seed)
    centers = rng.uniform(-3, 3, (9, d))
    x = (centers[rng.integers(0, 9, N)] + rng.uniform(-1.2e-3, 1.2e-3, (N, d))).astype(np.float32)
    f = np.round(rng.normal(0, 1, N), 1).astype(np.float32)
    stuck = rng.random(N) < 0.7
    return x, f, stuck


def _context_dedup(x, f, stuck, d, eps):
    N = x.shape[0]
    prob = I.small_mixture(d, 2, N, seed=30)
    model = U.open_ctx(prob, M.Params(eps_dup=eps))
    st = M.new_state(x, 4)
    st.f = f.astype(np.float64)
    st.stuck = stuck
    U.write_state(model, prob, st)
    model.run_phase(0, CH.PHASE_DEDUP)
    rem = CH.unpack_bits(model.get(0, CH.FIELD_REMOVED), N)
    k = model.counters(0)["k_lost"]
    model.close()
    return rem, k


def _noalloc_dedup(lib, x, f, stuck, d, eps, stream):
    import torch
    N = x.shape[0]
    xd = torch.from_numpy(x).cuda()
    fd = torch.from_numpy(f).cuda()
    sd = torch.from_numpy(CH.pack_bits(stuck).view(np.int32)).cuda()
    rd = torch.full(((N + 31) // 32,), -1, dtype=torch.int32, device="cuda")   # garbage: the call clears it
    kd = torch.full((1,), -7, dtype=torch.int32, device="cuda")
    torch.cuda.synchronize()
    st = lib.chisao_dedup_noalloc(xd.data_ptr(), d, N, fd.data_ptr(), sd.data_ptr(), eps, rd.data_ptr(),
                                  kd.data_ptr(), C.c_void_p(stream.cuda_stream))
    assert st == CH.OK
    stream.synchronize()
    rem = CH.unpack_bits(rd.cpu().numpy().view(np.uint32), N)
    return rem, int(kd.cpu().item())


@pytest.mark.parametrize("d", [3, 64])
def test_noalloc_dedup_matches_context_path_twice(d):
    import torch
    U.ensure_built()
    lib = CH.library()
    stream = torch.cuda.Stream()
    eps = 1e-3
    # two calls in a row with different inputs (the second one larger), sharing the scratch
    for seed, N in ((1, 2500), (2, 5001)):
        x, f, stuck = _case(seed + d, N, d)
        rem_ctx, k_ctx = _context_dedup(x, f, stuck, d, eps)
        rem_na, k_na = _noalloc_dedup(lib, x, f, stuck, d, eps, stream)
        np.testing.assert_array_equal(rem_na, rem_ctx)
        assert k_na == k_ctx == rem_ctx.sum()
        np.testing.assert_array_equal(rem_na, M.dedup(x, f, stuck, eps, dtype=np.float32))


def test_noalloc_dedup_rejects_oversize_and_bad_args():
    U.ensure_built()
    lib = CH.library()
    big = CH.library().chisao_dedup_noalloc(None, 3, (1 << 18) + 1, None, None, 1e-3, None, None, None)
    assert big == CH.ERR_CAPACITY
    assert lib.chisao_dedup_noalloc(None, 65, 10, None, None, 1e-3, None, None, None) == CH.ERR_ARG
    assert lib.chisao_dedup_noalloc(None, 3, 10, None, None, 1e-3, None, None, None) == CH.ERR_ARG
