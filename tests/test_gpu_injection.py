"""GPU parity with factor injection: the oracle's own patch and coarse inverses loaded
into the context (als_load_patch_inverses, als_load_coarse_inverse), so that the parity
of the smoother and of whole cycles is measured apart from the factorisations.

Without injection the two sides' inverses of an ill-conditioned patch differ by about
cond(A_v) eps (two different Cholesky/sweep roundings), which at DR 1e8 and gamma 1e4
(cond ~ 1e12) swamps the 1e-12 bar.  With identical inverses only the order of the
floating-point sums differs."""
import numpy as np
import pytest

from gpu_helpers import context, dev, host, oracle, random_free, rel, sinker, torch  # noqa: F401
from injection import inject, library_patch_inverses, load_into, packed_by_diagonals, unpack_by_diagonals

pytestmark = pytest.mark.gpu

from paper_2107_00820_gb300 import alstokes as A  # noqa: E402


@pytest.mark.parametrize("d,n,gamma,dr", [(2, 16, 1e2, 1e3), (2, 16, 1e4, 1e8), (3, 4, 1e4, 1e8)])
@pytest.mark.parametrize("prec", [A.ALS_PREC_FP64, A.ALS_PREC_FP32])
def test_smoother_apply_with_the_oracle_inverses(d, n, gamma, dr, prec):
    """The smoother output with the oracle's inverses matches the oracle's
    sum_v I_v A_v^-1 I_v^T r entry by entry within 1e-12 (FP64) of sum |terms|, at any
    contrast and gamma (DR 1e8, gamma 1e4 included), and within the FP32 rounding in FP32
    (the FP32 copies are rounded from the injected FP64 ones)."""
    from oracle.mg import all_vertices, star_dofs
    pb = sinker(d, n, 2, gamma, dr=dr, seed=37)
    H = oracle(pb, smoother="richardson", steps=1)
    inv0 = inject(H)
    full = library_patch_inverses(H, 1)
    np_ = d * 3 ** d
    fp64 = prec == A.ALS_PREC_FP64
    dt = torch.float64 if fp64 else torch.float32
    ctx = context(pb)
    load_into(ctx, H, inv0)
    if not fp64:
        packed = packed_by_diagonals(full, np_).astype(np.float32).astype(np.float64)
        full = np.stack([unpack_by_diagonals(pv, np_) for pv in packed])
    lv = H.levels[1]
    r = np.random.default_rng(38).standard_normal(lv.mesh.nu)
    r[lv.bdof] = 0.0
    if not fp64:
        r = r.astype(np.float32).astype(np.float64)
    ref, scale = np.zeros_like(r), np.zeros_like(r)
    NB = 3 ** d
    offs = np.array([[o % 3, (o // 3) % 3, o // 9][:d] for o in range(NB)]) - 1
    for v, F in zip(all_vertices(lv.mesh), full):
        idx = star_dofs(lv.mesh, v)
        g = 2 * v + offs
        free = np.all(g > 0, axis=1) & np.all(g < np.array(lv.mesh.nn) - 1, axis=1)
        keep = [a * NB + o for a in range(d) for o in range(NB) if free[o]]
        S = F[np.ix_(keep, keep)]
        ref[idx] += S @ r[idx]
        scale[idx] += np.abs(S) @ np.abs(r[idx])
    z = torch.full((lv.mesh.nu,), float("nan"), dtype=dt, device="cuda")
    ctx.star_smooth(1, dev(r, dt), z, prec)
    err = np.abs(host(z) - ref)
    tol = 1e-12 if fp64 else 200 * 2.0 ** -24
    assert np.all(err <= tol * scale + 1e-300), np.max(err / np.maximum(scale, 1e-300))
