"""The optional bfloat16 storage of the FP32 cycle's star inverses (options.store =
ALS_STORE_BF16): the smoother with the oracle's inverses injected, against the oracle's
star products on the same inverses rounded to bfloat16 (to nearest, from FP64), entry by
entry at FP32 rounding; and the mixed solve: a few FGMRES iterations more at mild
contrast, still a good preconditioner with the P2 pairing at DR 1e8 in 2D, no convergence
with the P1 pairing at DR 1e8 (the behaviour the option's documentation states)."""
import numpy as np
import pytest

from gpu_helpers import context, dev, host, oracle, sinker, torch  # noqa: F401
from injection import inject, library_patch_inverses, load_into, packed_by_diagonals, unpack_by_diagonals
from oracle.stokes import StokesSolver

pytestmark = pytest.mark.gpu

from paper_2107_00820_gb300 import alstokes as A  # noqa: E402


def to_bfloat16(x):
    """Round to the nearest bfloat16 (8 significant bits), ties to even, from float64."""
    m, e = np.frexp(np.asarray(x, dtype=np.float64))
    return np.ldexp(np.rint(m * 256.0) / 256.0, e)


def test_bfloat16_rounding_helper():
    assert to_bfloat16(1.0) == 1.0 and to_bfloat16(-3.0) == -3.0
    assert to_bfloat16(1.0 + 2.0 ** -8) == 1.0                   # a tie, to even
    assert to_bfloat16(1.0 + 3 * 2.0 ** -8) == 1.0 + 2.0 ** -6   # a tie, to even (up)
    assert to_bfloat16(1.0 + 2.0 ** -8 + 2.0 ** -20) == 1.0 + 2.0 ** -7
    x = np.random.default_rng(1).standard_normal(1000)
    assert np.all(np.abs(to_bfloat16(x) - x) <= 2.0 ** -8 * np.abs(x))   # half an ulp of 8 bits
    # PyTorch's float32 -> bfloat16 conversion (round to nearest even) on float32 inputs
    x = x.astype(np.float32).astype(np.float64)
    tb = torch.tensor(x, dtype=torch.float32).to(torch.bfloat16).to(torch.float64).numpy()
    assert np.array_equal(tb, to_bfloat16(x))


@pytest.mark.parametrize("d,n,gamma,dr", [(2, 16, 1e2, 1e3), (2, 16, 1e4, 1e8), (3, 4, 1e2, 1e4)])
def test_smoother_with_bfloat16_inverses(d, n, gamma, dr):
    from oracle.mg import all_vertices, star_dofs
    pb = sinker(d, n, 2, gamma, dr=dr, seed=41)
    H = oracle(pb, smoother="richardson", steps=1)
    inv0 = inject(H)
    full = library_patch_inverses(H, 1)
    np_ = d * 3 ** d
    ctx = context(pb, store=A.ALS_STORE_BF16)
    load_into(ctx, H, inv0)
    packed = to_bfloat16(packed_by_diagonals(full, np_))
    full = np.stack([unpack_by_diagonals(pv, np_) for pv in packed])
    lv = H.levels[1]
    r = np.random.default_rng(42).standard_normal(lv.mesh.nu)
    r[lv.bdof] = 0.0
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
    z = torch.full((lv.mesh.nu,), float("nan"), dtype=torch.float32, device="cuda")
    ctx.star_smooth(1, dev(r, torch.float32), z, A.ALS_PREC_FP32)
    err = np.abs(host(z) - ref)
    assert np.all(err <= 200 * 2.0 ** -24 * scale + 1e-300), np.max(err / np.maximum(scale, 1e-300))
    # and not the FP32 inverses: the bfloat16 rounding is visible in the output
    z32 = torch.zeros_like(z)
    ctx32 = context(pb)
    load_into(ctx32, H, inv0)
    ctx32.star_smooth(1, dev(r, torch.float32), z32, A.ALS_PREC_FP32)
    assert np.max(np.abs(host(z32) - host(z))) > 1e-4 * np.max(np.abs(host(z32)))


def test_mixed_solve_with_bfloat16_stars_at_mild_contrast():
    """DR 1e4, gamma 10: the bfloat16 cycle costs a few FGMRES iterations over FP32
    storage (17 -> 20 here) and meets the tolerance in the true residual."""
    pb = sinker(2, 32, 3, 10.0, dr=1e4, seed=43)
    s = StokesSolver(oracle(pb))
    _, _, i32 = context(pb, mode=A.ALS_MODE_MIXED, rtol=1e-8).solve(pb.f, pb.u_bc)
    u, p, i16 = context(pb, mode=A.ALS_MODE_MIXED, rtol=1e-8, store=A.ALS_STORE_BF16).solve(pb.f, pb.u_bc)
    assert i16.converged and i16.iterations <= i32.iterations + 4, (i16.iterations, i32.iterations)
    b, uD = s.rhs(pb.f, pb.u_bc)
    res = np.linalg.norm(b - s.matvec(np.concatenate([u - uD, p]))) / np.linalg.norm(b)
    assert res <= 1.5e-8


def test_bfloat16_stars_with_p2_at_extreme_contrast():
    """With the P2 pairing (W = M_p(1/mu)) the bfloat16 cycle stays a good preconditioner at
    DR 1e8 and gamma 1e3: a few iterations over FP32 storage, the tolerance met in the
    true residual."""
    pb = sinker(2, 32, 3, 1e3, dr=1e8, seed=44)
    s = StokesSolver(oracle(pb, W="Mp_mu"), schur="P2")
    opts = dict(mode=A.ALS_MODE_MIXED, rtol=1e-8, schur=A.ALS_SCHUR_P2)
    _, _, i32 = context(pb, **opts).solve(pb.f, pb.u_bc)
    u, p, i16 = context(pb, store=A.ALS_STORE_BF16, **opts).solve(pb.f, pb.u_bc)
    assert i32.converged and i16.converged and i16.iterations <= i32.iterations + 4, (i16.iterations, i32.iterations)
    b, uD = s.rhs(pb.f, pb.u_bc)
    res = np.linalg.norm(b - s.matvec(np.concatenate([u - uD, p]))) / np.linalg.norm(b)
    assert res <= 1.5e-8


def test_bfloat16_stars_lose_the_p1_cycle_at_high_contrast():
    """With the P1 pairing (W = M_p) at DR 1e8 the bfloat16 cycle stops being a useful
    preconditioner: no convergence to 1e-8 in three times the iterations FP32 storage
    needs (the limit the option's documentation states)."""
    pb = sinker(3, 8, 2, 10.0, dr=1e8, seed=45)
    _, _, i32 = context(pb, mode=A.ALS_MODE_MIXED, rtol=1e-8).solve(pb.f, pb.u_bc)
    assert i32.converged
    ctx = context(pb, mode=A.ALS_MODE_MIXED, rtol=1e-8, maxit=3 * i32.iterations, store=A.ALS_STORE_BF16)
    _, _, i16 = ctx.solve(pb.f, pb.u_bc, check=False)
    assert not i16.converged, (i16.iterations, i32.iterations)
