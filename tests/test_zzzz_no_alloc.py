"""The allocation-free star smoother against the context's smoother.

als_star_smooth_static serves callers that may not allocate device memory
while they smooth (a real-time loop whose device memory is budgeted up front,
a plugin whose host framework owns the allocator, code that cannot afford an
allocation's implicit synchronisation): its scratch is a fixed array inside the
library.  It must give the same z as als_star_smooth on the same patch
inverses, call after call (the array keeps the previous call's contents, which
must not leak into the next result).  This file is collected last, so that a
run that stops at the first failure has run every other test before it.
"""
import numpy as np
import pytest

from gpu_helpers import context, dev, host, rel, sinker, torch  # noqa: F401

pytestmark = pytest.mark.gpu

from paper_2107_00820_gb300 import alstokes as A  # noqa: E402


def _packed_by_diagonals(full, np_):
    stride = ((np_ * (np_ + 1) // 2) + 3) & ~3
    out = np.zeros((len(full), stride))
    for v, F in enumerate(full):
        pos = 0
        for t in range(np_):
            out[v, pos:pos + np_ - t] = np.diagonal(F, offset=t)
            pos += np_ - t
    return out


@pytest.mark.parametrize("d,n,prec", [(2, 16, A.ALS_PREC_FP64), (2, 16, A.ALS_PREC_FP32),
                                      (3, 4, A.ALS_PREC_FP64), (3, 4, A.ALS_PREC_FP32)])
def test_static_scratch_smoother_matches_context_smoother(d, n, prec):
    pb = sinker(d, n, 2, 1e2, dr=1e3, seed=31)
    ctx = context(pb)
    nverts = (n + 1) ** d
    np_ = d * 3 ** d
    full = [ctx.patch_inverse(1, v) for v in range(nverts)]
    dt = torch.float64 if prec == A.ALS_PREC_FP64 else torch.float32
    inv = dev(_packed_by_diagonals(full, np_), dt)
    stream = torch.cuda.current_stream().cuda_stream
    tol = 1e-11 if prec == A.ALS_PREC_FP64 else 1e-4       # the smoother tolerances of the parity tests
    for seed in (1, 2):                                     # two calls in a row share the scratch array
        r = np.random.default_rng(seed).standard_normal(ctx.nu())
        r_d = dev(r, dt)
        z_ctx = torch.zeros(ctx.nu(), dtype=dt, device="cuda")
        ctx.star_smooth(1, r_d, z_ctx, prec)
        z_st = torch.full((ctx.nu(),), float("nan"), dtype=dt, device="cuda")
        A.als_star_smooth_static(d, [n] * d, prec, inv, r_d, z_st, stream)
        torch.cuda.synchronize()
        assert rel(host(z_st), host(z_ctx)) <= tol


def test_static_scratch_rejects_meshes_beyond_its_size():
    big = torch.zeros(8, dtype=torch.float64, device="cuda")
    with pytest.raises(A.ALSError) as e:
        A.als_star_smooth_static(3, [64, 64, 64], A.ALS_PREC_FP64, big, big, big)
    assert e.value.status == A.ALS_EINVAL
