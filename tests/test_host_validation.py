"""Host-side argument checks of the C ABI, on the CPU (no GPU is touched).

als_create validates the mesh, the coefficients and every option before it creates a
stream or allocates anything, so these run anywhere the library loads: each invalid
argument is refused with ALS_EINVAL and a message that names it, readable through
als_last_error(NULL) after the context is gone; every entry point refuses a NULL
context; the documented defaults are what als_default_options fills in."""
import ctypes

import numpy as np
import pytest

from paper_2107_00820_gb300 import alstokes as A


@pytest.fixture(scope="module")
def lib():
    from paper_2107_00820_gb300 import build as b
    if not b.up_to_date():
        import os
        if not os.path.exists("/usr/local/cuda/bin/nvcc"):
            pytest.skip("nvcc not available to build the library")
        b.build()
    return A.load()


def test_default_options(lib):
    o = A.als_options()
    lib.als_default_options(ctypes.byref(o))
    assert (o.smoother, o.sweeps, o.transfer, o.schur, o.mode) == \
        (A.ALS_SMOOTH_GMRES, 5, A.ALS_TRANSFER_ROBUST, A.ALS_SCHUR_P1, A.ALS_MODE_FP64)
    assert (o.cycle, o.fact, o.maxit) == (A.ALS_CYCLE_V, A.ALS_FACT_FULL, 300)
    assert o.rtol == 1e-8 and o.tau == 0.0          # tau 0: 2^-d chosen at create
    assert o.setup == A.ALS_SETUP_AUTO
    assert (o.order, o.store) == (2, A.ALS_STORE_FP32)


@pytest.mark.parametrize("args,kw,words", [
    ((4, (4, 4, 4), 1), {}, "dim"),
    ((2, 4, 0), {}, "levels"),
    ((2, 4, 13), {}, "levels"),
    ((2, 6, 3), {}, "divisible"),
    ((2, 4, 3), {}, "coarse cells"),
    ((2, 4, 1), {"sweeps": 0}, "sweeps"),
    ((2, 4, 1), {"sweeps": 65}, "sweeps"),
    ((2, 4, 1), {"maxit": 0}, "maxit"),
    ((2, 4, 1), {"schur": 2}, "Schur"),
    ((2, 4, 1), {"cycle": 2}, "cycle"),
    ((2, 4, 1), {"fact": 4}, "factorisation"),
    ((2, 4, 1), {"smoother": 2}, "smoother"),
    ((2, 4, 1), {"transfer": 2}, "transfer"),
    ((2, 4, 1), {"mode": 2}, "mode"),
    ((2, 4, 1), {"setup": 2}, "setup"),
    ((2, 4, 1), {"store": 2}, "star storage"),
    ((2, 4, 1), {"store": 1, "order": 3}, "bfloat16 star storage"),
    ((3, 1024, 2), {}, "too large"),
    ((2, 46340, 2), {}, "too large"),
])
def test_create_rejects_invalid_arguments(lib, args, kw, words):
    d, n, levels = args
    mu = [np.zeros(1)] * levels           # never read: the arguments are refused first
    with pytest.raises(A.ALSError) as e:
        A.Context(d, n, levels, mu, 1.0, **kw)
    assert e.value.status == A.ALS_EINVAL
    assert words in str(e.value), str(e.value)
    assert words in lib.als_last_error(None).decode()


@pytest.mark.parametrize("d", [2, 3])
def test_order_three_refuses_tensor_coefficients(lib, d):
    """Order 3 is built for scalar viscosity in 2D and 3D: tensor coefficients are refused
    before any device work (the arrays are never read)."""
    mu = [np.zeros(1)] * 2
    with pytest.raises(A.ALSError) as e:
        A.Context(d, 4, 2, mu, 1.0, mu_eff=mu, order=3)
    assert e.value.status == A.ALS_EINVAL and "scalar viscosity" in str(e.value), str(e.value)


@pytest.mark.parametrize("gamma", [-1.0, float("nan"), float("inf")])
def test_create_rejects_invalid_gamma(lib, gamma):
    with pytest.raises(A.ALSError) as e:
        A.Context(2, 4, 1, [np.ones((16, 9))], gamma)
    assert e.value.status == A.ALS_EINVAL and "gamma" in str(e.value)


def test_create_rejects_tensor_without_mu_eff(lib):
    mesh = A.als_mesh(2, (ctypes.c_int * 3)(4, 4, 1), 1)
    qp = (ctypes.c_void_p * 1)(ctypes.c_void_p(1))
    coeff = A.als_coeff(A.ALS_COEFF_TENSOR, qp, None)
    out = ctypes.c_void_p()
    st = lib.als_create(ctypes.byref(mesh), ctypes.byref(coeff), 1.0, None, None, ctypes.byref(out))
    assert st == A.ALS_EINVAL and out.value is None
    assert "mu_eff" in lib.als_last_error(None).decode()
    coeff = A.als_coeff(7, qp, None)
    assert lib.als_create(ctypes.byref(mesh), ctypes.byref(coeff), 1.0, None, None, ctypes.byref(out)) == A.ALS_EINVAL
    assert "kind" in lib.als_last_error(None).decode()
    assert lib.als_create(ctypes.byref(mesh), None, 1.0, None, None, ctypes.byref(out)) == A.ALS_EINVAL
    assert lib.als_create(ctypes.byref(mesh), ctypes.byref(coeff), 1.0, None, None, None) == A.ALS_EINVAL


def test_batch_create_names_the_failing_instance(lib):
    meshes = (A.als_mesh * 2)(A.als_mesh(2, (ctypes.c_int * 3)(4, 4, 1), 1),
                              A.als_mesh(5, (ctypes.c_int * 3)(4, 4, 1), 1))
    qp = (ctypes.c_void_p * 1)(ctypes.c_void_p(1))
    coeffs = (A.als_coeff * 2)(A.als_coeff(A.ALS_COEFF_SCALAR, qp, None), A.als_coeff(A.ALS_COEFF_SCALAR, qp, None))
    gammas = (ctypes.c_double * 2)(1.0, 1.0)
    out = ctypes.c_void_p()
    # instance 0 is valid but would need a GPU: give instance 0 an invalid gamma instead
    gammas[0] = -1.0
    st = lib.als_batch_create(2, meshes, coeffs, gammas, None, None, ctypes.byref(out))
    assert st == A.ALS_EINVAL and out.value is None
    msg = lib.als_last_error(None).decode()
    assert msg.startswith("instance 0") and "gamma" in msg
    assert lib.als_batch_create(0, meshes, coeffs, gammas, None, None, ctypes.byref(out)) == A.ALS_EINVAL


def test_every_entry_point_refuses_a_null_context(lib):
    N = None
    d, i, ll = ctypes.c_double(), ctypes.c_int(), ctypes.c_longlong()
    calls = {
        "als_destroy": (N,), "als_apply_agamma": (N, 0, 0, N, N), "als_vcycle": (N, 0, N, N),
        "als_star_smooth": (N, 1, 0, N, N), "als_prolong": (N, 1, 0, N, N), "als_restrict": (N, 1, 0, N, N),
        "als_coarse_solve": (N, 0, N, N), "als_apply_stokes": (N, N, N, N, N),
        "als_patch_inverse": (N, 0, 0, N), "als_solve": (N, N, N, N, N, N, N),
        "als_update_coefficients": (N, N), "als_profile": (N, 1),
        "als_profile_read": (N, ctypes.byref(d), ctypes.byref(ll)),
        "als_profile_read_kernel": (N, 0, ctypes.byref(d), ctypes.byref(ll)),
        "als_autotune_info": (N, 1, ctypes.byref(i), N), "als_set_patch_kernel": (N, 1, 0),
        "als_batch_destroy": (N,), "als_batch_context": (N, 0, N), "als_batch_vcycle": (N, 0, N, N),
        "als_batch_solve": (N, N, N, N, N, N, N), "als_measure_fma_peaks": (N, N, N),
        "als_load_patch_inverses": (N, 1, N), "als_load_coarse_inverse": (N, N),
        "als_set_wait_limit": (N, 0), "als_solve_history": (N, N, 0, ctypes.byref(i)),
        "als_batch_set_mode": (N, 0), "als_batch_get_mode": (N, ctypes.byref(i)),
        "als_batch_merged_plan": (N, ctypes.byref(i), ctypes.byref(i), N, N), "als_batch_set_grouping": (N, 0),
        "als_batch_merged_tune": (N, 0, 1, ctypes.byref(i), ctypes.byref(i), N, N),
    }
    for name, args in calls.items():
        assert getattr(lib, name)(*args) == A.ALS_EINVAL, name
    assert lib.als_star_smooth_static(4, N, 1, N, N, N, N) == A.ALS_EINVAL
    assert lib.als_batch_last_error(None) == b"null batch"


def test_binding_marshalling_checks(lib):
    """The binding's own argument checks, before any call crosses the ABI: contiguous
    arrays only, the dtype that matches the precision, CUDA tensors for the device entry
    points, known option names, and readable status names in its errors."""
    x = np.zeros((4, 4))
    assert A._ptr(None) is None and A._ptr(x).value == x.ctypes.data
    with pytest.raises(ValueError):
        A._ptr(x[:, ::2])
    with pytest.raises(TypeError):
        A._ptr([1.0, 2.0])
    A._check_dtype(np.zeros(2), A.ALS_PREC_FP64)
    A._check_dtype(np.zeros(2, np.float32), A.ALS_PREC_FP32)
    with pytest.raises(TypeError):
        A._check_dtype(np.zeros(2, np.float32), A.ALS_PREC_FP64)
    with pytest.raises(TypeError):
        A._check_dtype(np.zeros(2), A.ALS_PREC_FP32)
    with pytest.raises(TypeError):
        A._cuda_tensor(np.zeros(2))
    torch = pytest.importorskip("torch")
    with pytest.raises(TypeError):
        A._cuda_tensor(torch.zeros(2))                         # a CPU tensor is refused too
    with pytest.raises(ValueError):
        A._ptr(torch.zeros(4, 4).t())
    o = A.default_options(sweeps=3, mode=A.ALS_MODE_MIXED)
    assert o.sweeps == 3 and o.mode == A.ALS_MODE_MIXED
    with pytest.raises(KeyError):
        A.default_options(no_such_option=1)
    assert str(A.ALSError(A.ALS_ENOTSPD, "patch 7")) == "ALS_ENOTSPD: patch 7"


@pytest.mark.parametrize("n", [[2 ** 31 - 2] * 2, [4097, 4], [0, 4], [-3, 4], [64, 64, 64]])
def test_static_smoother_refuses_sizes_before_any_launch(lib, n):
    """The allocation-free smoother bounds every axis before it forms a product (no
    wrap-around for huge n) and refuses meshes whose per-patch outputs exceed its fixed
    scratch array; it returns ALS_EINVAL before touching the GPU (here: none)."""
    dim = len(n)
    arr = (ctypes.c_int * 3)(*(n + [1] * (3 - dim)))
    fake = ctypes.c_void_p(16)                      # never dereferenced: refused first
    for prec in (A.ALS_PREC_FP64, A.ALS_PREC_FP32):
        assert lib.als_star_smooth_static(dim, arr, prec, fake, fake, fake, None) == A.ALS_EINVAL


def test_static_smoother_binding_checks(lib):
    """The binding hands the allocation-free smoother only CUDA tensors of the precision's
    dtype that are long enough for the mesh (host arrays, CPU tensors, the wrong dtype or
    short buffers are refused before the call)."""
    torch = pytest.importorskip("torch")
    with pytest.raises(TypeError):
        A.als_star_smooth_static(2, [4, 4], A.ALS_PREC_FP64, np.zeros(8), np.zeros(8), np.zeros(8))
    with pytest.raises(TypeError):
        A.als_star_smooth_static(2, [4, 4], A.ALS_PREC_FP64, torch.zeros(8), torch.zeros(8), torch.zeros(8))


@pytest.mark.parametrize("dim,order,n,levels", [(2, 2, (8, 8), 2), (3, 2, (4, 4, 4), 2), (2, 3, (8, 8), 2),
                                                (3, 3, (4, 4, 4), 2)])
def test_injection_binding_checks_length_and_dtype(dim, order, n, levels):
    """Factor injection copies exactly nverts x stride (patches) and nfree^2 (coarse)
    doubles from the caller's buffer, so the binding refuses a short array, FP32 data, or
    a level without patches before any call crosses the ABI (the context here has no
    library handle: reaching the ABI would raise AttributeError instead)."""
    ctx = A.Context.__new__(A.Context)
    ctx.dim, ctx.n, ctx.levels = dim, n, levels
    ctx.options = A.default_options(order=order)
    np_ = dim * (2 * order - 1) ** dim
    assert ctx.patch_dofs() == {(2, 2): 18, (3, 2): 81, (2, 3): 50, (3, 3): 375}[(dim, order)]
    stride = (np_ * (np_ + 1) // 2 + 3) // 4 * 4
    need = int(np.prod([v + 1 for v in n])) * stride
    with pytest.raises(ValueError):
        ctx.load_patch_inverses(1, np.zeros(need - 1))
    with pytest.raises(TypeError):
        ctx.load_patch_inverses(1, np.zeros(need, np.float32))
    with pytest.raises(ValueError):
        ctx.load_patch_inverses(0, np.zeros(need))
    nf = dim * int(np.prod([order * v // 2 - 1 for v in n]))
    assert ctx.coarse_free_dofs() == nf
    with pytest.raises(ValueError):
        ctx.load_coarse_inverse(np.zeros(nf * nf - 1))
    with pytest.raises(TypeError):
        ctx.load_coarse_inverse(np.zeros(nf * nf, np.float32))
