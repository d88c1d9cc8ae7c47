"""The allocation-free star smoother against the context's smoother.

als_star_smooth_static serves callers that may not allocate device memory
while they smooth (inside a global-mode stream capture, in a pre-budgeted
real-time loop, under a host framework that owns the allocator): its
scratch is a fixed array inside the library.  It must give the same z as
als_star_smooth on the same patch inverses, call after call (the array keeps
the previous call's contents, which must not leak into the next result).
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


def _oracle_inverses(H, lvl):
    """The oracle's star-patch inverses in the library's layout: per vertex (x-fastest) the
    full d 3^d matrix, component-major, star offsets x-fastest, identity at absent and
    boundary nodes; the oracle's upper triangle mirrored, which is what the packed
    storage keeps."""
    from oracle.mg import all_vertices
    m = H.levels[lvl].mesh
    d, NB = m.d, 3 ** m.d
    verts = all_vertices(m)
    offs = np.array([[o % 3, (o // 3) % 3, o // 9][:d] for o in range(NB)]) - 1
    full = np.tile(np.eye(d * NB), (len(verts), 1, 1))
    for ids, _, _, inv in H.patches[lvl].groups.values():
        for i, X in zip(ids, inv):
            g = 2 * verts[i] + offs
            free = np.all(g > 0, axis=1) & np.all(g < np.array(m.nn) - 1, axis=1)
            keep = [a * NB + o for a in range(d) for o in range(NB) if free[o]]
            full[i][np.ix_(keep, keep)] = np.triu(X) + np.triu(X, 1).T
    return full


@pytest.mark.parametrize("d,n,gamma,dr", [(2, 16, 1e2, 1e3), (2, 16, 1e4, 1e8), (3, 4, 1e4, 1e8)])
@pytest.mark.parametrize("prec", [A.ALS_PREC_FP64, A.ALS_PREC_FP32])
def test_smoother_apply_with_the_oracle_inverses(d, n, gamma, dr, prec):
    """Factor injection: the oracle's own patch inverses loaded into the allocation-free
    smoother separate the apply from the factorisation.  With identical inverses the only
    difference left is the summation order, so the smoother output matches the oracle's
    sum_v I_v A_v^-1 I_v^T r entry by entry within 1e-12 (FP64) of sum |terms|, at any
    contrast and gamma (DR 1e8, gamma 1e4 included), and within the FP32 rounding in FP32."""
    from gpu_helpers import oracle
    from oracle.mg import all_vertices, star_dofs
    pb = sinker(d, n, 2, gamma, dr=dr, seed=37)
    H = oracle(pb, smoother="richardson", steps=1)
    full = _oracle_inverses(H, 1)
    np_ = d * 3 ** d
    fp64 = prec == A.ALS_PREC_FP64
    dt = torch.float64 if fp64 else torch.float32
    packed = _packed_by_diagonals(full, np_)
    if not fp64:
        packed = packed.astype(np.float32).astype(np.float64)
        full = np.stack([_unpack_by_diagonals(pv, np_) for pv in packed])
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
    stream = torch.cuda.current_stream().cuda_stream
    A.als_star_smooth_static(d, [n] * d, prec, dev(packed, dt), dev(r, dt), z, stream)
    torch.cuda.synchronize()
    err = np.abs(host(z) - ref)
    tol = 1e-12 if fp64 else 200 * 2.0 ** -24
    assert np.all(err <= tol * scale + 1e-300), np.max(err / np.maximum(scale, 1e-300))


def _unpack_by_diagonals(pv, np_):
    F = np.zeros((np_, np_))
    pos = 0
    for t in range(np_):
        k = np_ - t
        F[np.arange(k), np.arange(t, np_)] = pv[pos:pos + k]
        F[np.arange(t, np_), np.arange(k)] = pv[pos:pos + k]
        pos += k
    return F
