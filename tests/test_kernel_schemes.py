"""Host checks of the index schemes of the order-3 star kernels (csrc/qk3.cu, csrc/qk.cu) and of
the shared-memory layouts of the order-2 3D cell kernel (csrc/apply_lines.cuh), restated
in NumPy: the enumeration of an upper triangle by paired rows, the symmetric block
Gauss-Jordan elimination on the upper triangle with the sign invariant
M_ji = s_i s_j M_ij, the product over wrapped rows W_t[i] = A(i, (i + t) mod N) (odd N in 3D, even in 2D),
and the paired-diagonal product of the FP64 kernel.  Each restates the kernel's loop
structure (not its arithmetic order) and compares with the plain dense result; a wrong
index, sign or bound fails it.  CPU only; these emulate kernels, they are not the oracle."""
import numpy as np
import pytest


def tri_entry(N, e):
    half = (N - 1) // 2
    p, off = divmod(e, N + 1)
    if p < half:
        if off < N - p:
            return p, p + off
        i = N - 1 - p
        return i, i + off - (N - p)
    return half, half + off


def diag_start(n, t):
    return t * n - (t * (t - 1)) // 2


@pytest.mark.parametrize("N", [27, 375, 5])
def test_triangle_enumeration_covers_each_entry_once(N):
    seen = [tri_entry(N, e) for e in range(N * (N + 1) // 2)]
    assert len(set(seen)) == len(seen) == N * (N + 1) // 2
    assert all(0 <= i <= j < N for i, j in seen)
    # consecutive e walk along a row (coalesced rows of the workspace)
    steps = sum(1 for a, b in zip(seen, seen[1:]) if a[0] == b[0] and b[1] == a[1] + 1)
    assert steps >= len(seen) - 2 * N


def symmetric_block_gauss_jordan(A, BB):
    """The kernel's passes on the upper triangle only: X_x = M(min(x, K), max(x, K)),
    Y = Dk X, M_ij -= sigma_j X_i . Y_j (sigma_j = -1 for j < k0), M_iK = -Y_i (i < k0),
    M_Kj = Y_j (j beyond K), M_KK = Dk."""
    N = A.shape[0]
    M = np.triu(A).astype(np.float64)
    for k0 in range(0, N, BB):
        b = min(BB, N - k0)
        K = np.arange(k0, k0 + b)
        Dk = np.linalg.inv(np.array([[M[min(m, l), max(m, l)] for l in K] for m in K]))
        X = np.zeros((N, b))
        for x in range(N):
            if k0 <= x < k0 + b:
                continue
            for li, k in enumerate(K):
                X[x, li] = M[x, k] if x < k else M[k, x]
        Y = Dk @ X.T
        new = M.copy()
        for e in range(N * (N + 1) // 2):
            i, j = tri_entry(N, e)
            ik, jk = k0 <= i < k0 + b, k0 <= j < k0 + b
            if ik and jk:
                new[i, j] = Dk[i - k0, j - k0]
            elif jk:
                new[i, j] = -Y[j - k0, i]
            elif ik:
                new[i, j] = Y[i - k0, j]
            else:
                sigma = -1.0 if j < k0 else 1.0
                new[i, j] = M[i, j] - sigma * X[i] @ Y[:, j]
        M = new
    return M


@pytest.mark.parametrize("N,BB", [(37, 16), (27, 16), (75, 16), (33, 8)])
def test_symmetric_block_gauss_jordan_inverts(N, BB):
    rng = np.random.default_rng(N)
    B = rng.standard_normal((N, N))
    A = B @ B.T + N * np.eye(N)
    M = symmetric_block_gauss_jordan(A, BB)
    Ainv = np.linalg.inv(A)
    assert np.abs(np.triu(M) - np.triu(Ainv)).max() <= 1e-13 * np.abs(Ainv).max()


def test_symmetric_block_gauss_jordan_with_identity_rows():
    """Absent and Dirichlet star nodes enter as identity rows and columns: their entries of
    the inverse stay exactly those of the identity."""
    rng = np.random.default_rng(3)
    N, free = 37, np.ones(37, bool)
    free[[0, 5, 6, 20, 36]] = False
    B = rng.standard_normal((N, N))
    A = B @ B.T + N * np.eye(N)
    A[~free] = 0.0
    A[:, ~free] = 0.0
    A[~free, ~free] = 1.0
    M = symmetric_block_gauss_jordan(A, 16)
    U = np.triu(M)
    idx = np.flatnonzero(~free)
    assert np.all(U[np.ix_(idx, idx)] == np.triu(np.eye(len(idx))))
    mixed = np.not_equal.outer(free, free)      # one index free, the other not
    assert np.all(U[np.triu(mixed)] == 0.0)
    Ainv = np.linalg.inv(A)
    assert np.abs(U - np.triu(Ainv)).max() <= 1e-13 * np.abs(Ainv).max()


@pytest.mark.parametrize("N", [375, 7])
def test_wrapped_row_product(N):
    WT, WLD = (N + 1) // 2, (N + 4) // 4 * 4
    rng = np.random.default_rng(1)
    A = rng.standard_normal((N, N))
    A = A + A.T
    W = np.zeros((WT, WLD))
    for t in range(WT):
        for i in range(N):
            W[t, i] = A[i, (i + t) % N]
    assert WT * WLD >= N * (N + 1) // 2
    r = rng.standard_normal(N)
    r2 = np.concatenate([r, r])
    y = np.zeros(N)
    for t in range(WT):
        for i in range(N):
            y[i] += W[t, i] * r2[i + t]
            if t > 0:
                m = i - t + N if i - t < 0 else i - t
                y[i] += W[t, m] * r2[m]
    assert np.abs(y - A @ r).max() <= 1e-12 * np.abs(A).sum(1).max()


@pytest.mark.parametrize("N", [50, 8])
def test_wrapped_row_product_even_order(N):
    """Even N (the 2D order-3 stars, N = 50): rows t = 0..N/2, the row N/2 read once per
    row (it holds each pair {i, i + N/2} twice), the transposed term for 0 < t < N/2."""
    WT, WLD = N // 2 + 1, (N + 3) // 4 * 4
    rng = np.random.default_rng(N)
    A = rng.standard_normal((N, N))
    A = A + A.T
    W = np.zeros((WT, WLD))
    for t in range(WT):
        for i in range(N):
            W[t, i] = A[i, (i + t) % N]
    r = rng.standard_normal(N)
    r2 = np.concatenate([r, r])
    y = np.zeros(N)
    for t in range(WT):
        for i in range(N):
            y[i] += W[t, i] * r2[i + t]
            if 0 < t < N // 2:
                m = i - t + N if i - t < 0 else i - t
                y[i] += W[t, m] * r2[m]
    assert np.abs(y - A @ r).max() <= 1e-12 * np.abs(A).sum(1).max()


@pytest.mark.parametrize("N", [375, 9])
def test_paired_diagonal_product(N):
    """The FP64 star product over packed diagonals, steps t and N - t in one iteration."""
    rng = np.random.default_rng(N)
    A = rng.standard_normal((N, N))
    A = A + A.T
    S = np.concatenate([np.diag(A, t) for t in range(N)])
    r = rng.standard_normal(N)
    y = np.array([S[i] * r[i] for i in range(N)])
    for t in range(1, N // 2 + 1):
        u = N - t
        for i in range(N):
            a, b = i < u, i < t
            p1 = diag_start(N, t) + i if a else diag_start(N, u) + (i - u)
            p2 = diag_start(N, u) + i if b else diag_start(N, t) + (i - t)
            assert 0 <= p1 < len(S) and 0 <= p2 < len(S)
            y[i] += S[p1] * r[i + t if a else i - u] + S[p2] * r[i + u if b else i - t]
    assert np.abs(y - A @ r).max() <= 1e-12 * np.abs(A).sum(1).max()


@pytest.mark.parametrize("count", [1, 7, 81, 3648, 3649, 16641])
@pytest.mark.parametrize("sms", [152, 1])
def test_persistent_star_walk_with_prefetch(count, sms):
    """The 2D order-3 FP32 star kernel's walk: min(ceil(count / 8), 3 sms) blocks of 8 warps,
    warp item = block * 8 + w, then item + warps ...; the warp fetches its first star before
    the loop and, in each pass, the next star (if any) before it multiplies the current one.
    Every star is staged and multiplied exactly once, always from the fetch made one pass
    earlier; the 16-byte words of a star (1,352 floats) split over 32 lanes in 11 slots
    cover each word once."""
    WPB, NV = 8, 26 * 52 // 4
    blocks = max(1, min((count + 7) // 8, 3 * sms))
    nwarps = blocks * WPB
    done = []
    for b in range(blocks):
        for w in range(WPB):
            item = b * WPB + w
            if item >= count:
                continue
            held = item                    # fetch(item) before the loop
            while True:
                staged = held              # the registers go to shared memory
                nxt = item + nwarps
                if nxt < count:
                    held = nxt             # fetch(next), in flight during the products
                assert staged == item
                done.append(item)
                if nxt >= count:
                    break
                item = nxt
    assert sorted(done) == list(range(count))
    words = [lane + 32 * q for q in range((NV + 31) // 32) for lane in range(32) if lane + 32 * q < NV]
    assert sorted(words) == list(range(NV))


@pytest.mark.parametrize("N", [50, 8])
def test_wrapped_row_product_paired_rows(N):
    """The 2D order-3 FP32 kernel's pairing: lane j < N/2 owns rows j and j + N/2 and walks
    t = 0..N/2, taking row j at step t and row j + N/2 at step N/2 - t, which need the same
    two r values (r_(j+t) and r_(j-t mod N)); each row gets every forward term once and the
    transposed terms for 0 < step < N/2, so the product equals A r."""
    H, WLD = N // 2, (N + 3) // 4 * 4
    rng = np.random.default_rng(N + 1)
    A = rng.standard_normal((N, N))
    A = A + A.T
    W = np.zeros((H + 1, WLD))
    for t in range(H + 1):
        for i in range(N):
            W[t, i] = A[i, (i + t) % N]
    r = rng.standard_normal(N)
    r2 = np.concatenate([r, r])
    y = np.zeros(N)
    for j in range(H):
        acc0 = acc1 = 0.0
        for t in range(H + 1):
            a, b = r2[j + t], r2[j - t + N]
            assert 0 <= j + t < N and 0 <= j - t + N < 2 * N
            acc0 += W[t, j] * a
            if 0 < t < H:
                m = j - t + N if j - t < 0 else j - t
                acc0 += W[t, m] * b
                acc1 += W[H - t, j + t] * a
            acc1 += W[H - t, j + H] * b
        y[j], y[j + H] = acc0, acc1
    assert np.abs(y - A @ r).max() <= 1e-12 * np.abs(A).sum(1).max()


def _ofs_xy(m, c, x, y, z):
    return m * 81 + c * 9 + x + 27 * y + 3 * z


def _ofs_yz(m, c, x, y, z):
    return m * 81 + c * 9 + 3 * x + y + 27 * z


def _ofs_pt(m, c, x, y, z):
    return m * 81 + c * 27 + 3 * x + 9 * y + z


def test_line_kernel_stage_layouts_are_bank_conflict_free():
    """The 3D line-per-lane cell kernel: lane (c, b1, b2) = (lane / 9, lane % 3, lane / 3 % 3)
    of 27 in its line stages, lane = Gauss point (p % 3, p / 3 % 3, p / 9) in its point stage.
    Every shared-memory access of every stage (one instruction = one fixed array m and one
    fixed line position) puts the 27 lanes on 27 distinct 4-byte banks, as the layouts'
    comment states, and so do the staged outputs (lane * 3 + a).  The block write-out
    (thread (row, cell) = (tid / 8, tid % 8) of 216 reading its cell's three values of a
    row, cells 243 floats apart) is at most 2-way conflicted: 32 threads on 20 banks; a
    244-float stride would make it conflict-free."""
    lanes = [(ln // 9, (ln % 9) % 3, (ln % 9) // 3) for ln in range(27)]
    pts = [(p % 3, (p // 3) % 3, p // 9) for p in range(27)]
    accesses = []
    for m in range(3):
        for q in range(3):
            accesses += [
                [_ofs_xy(m, c, q, b1, b2) for c, b1, b2 in lanes],   # X write, X^T read
                [_ofs_xy(m, c, b1, q, b2) for c, b1, b2 in lanes],   # Y read, Y^T write
                [_ofs_yz(m, c, b1, q, b2) for c, b1, b2 in lanes],   # Y write, Y^T read
                [_ofs_yz(m, c, b1, b2, q) for c, b1, b2 in lanes],   # Z read, Z^T write
                [_ofs_pt(m, c, b1, b2, q) for c, b1, b2 in lanes],   # Z write, Z^T read
                [_ofs_pt(m, q, *p) for p in pts],                     # gradient read, flux write
            ]
    for a in range(3):
        accesses.append([ln * 3 + a for ln in range(27)])           # staged x-line outputs
    for addrs in accesses:
        assert len(set(addrs)) == 27 and len({x % 32 for x in addrs}) == 27
    for stride, worst in ((243, 2), (244, 1)):                       # block write-out, 216 threads
        for warp in range(27 * 8 // 32 + 1):
            tids = [t for t in range(32 * warp, 32 * warp + 32) if t < 27 * 8]
            for a in range(3):
                banks = [((t & 7) * stride + (t >> 3) * 3 + a) % 32 for t in tids]
                assert max(banks.count(b) for b in set(banks)) == worst


def _patch_out_index(nv, vx, vy, vz, i):
    """The row layout of the 3D star-patch outputs (csrc/common.cuh, patch_out_index)."""
    c, o = divmod(i, 27)
    ox, oy, oz = o % 3, (o // 3) % 3, o // 9
    row = ((c * 3 + oz) * 3 + oy) * (nv[1] * nv[2]) + vz * nv[1] + vy
    return row * (3 * nv[0]) + 3 * vx + ox


@pytest.mark.parametrize("n", [(4, 3, 5), (2, 2, 2)])
def test_fused_patch_gather_in_the_cell_kernel(n):
    """The 3D cell kernel's x-line input formed from the star-patch outputs (apply_lines.cuh,
    patch_line): lane (c, b1, b2) of cell (cx, cy, cz) sums, for the nodes 2cx + a of its
    x-line, the outputs of the <= 8 stars containing each node, read from the row layout as
    columns 3cx + 1 (a = 0), 3cx + 2 and 3cx + 3 (a = 1), 3cx + 4 (a = 2) of the rows of
    its <= 4 (y, z) taps; 0 at Dirichlet nodes.  That equals the direct sum over stars, and
    the owner rule (the cell with the node's lower corner, the last cell for the upper
    boundary) stores every node of the mesh exactly once."""
    nv = [v + 1 for v in n]
    nn = [2 * v + 1 for v in n]
    rng = np.random.default_rng(sum(n))
    star = rng.standard_normal((nv[0] * nv[1] * nv[2], 81))      # star outputs, patch dof order
    out = np.zeros(81 * nv[1] * nv[2] * 3 * nv[0] + 8)
    for vz in range(nv[2]):
        for vy in range(nv[1]):
            for vx in range(nv[0]):
                v = vx + nv[0] * (vy + nv[1] * vz)
                for i in range(81):
                    out[_patch_out_index(nv, vx, vy, vz, i)] = star[v, i]
    # direct sums: node (ni, nj, nk) of component c collects star v at offset o when
    # ni = 2 vx + ox - 1 (per axis); 0 on the boundary
    direct = np.zeros((3, nn[2], nn[1], nn[0]))
    for vz in range(nv[2]):
        for vy in range(nv[1]):
            for vx in range(nv[0]):
                v = vx + nv[0] * (vy + nv[1] * vz)
                for i in range(81):
                    c, o = divmod(i, 27)
                    ni, nj, nk = 2 * vx + o % 3 - 1, 2 * vy + (o // 3) % 3 - 1, 2 * vz + o // 9 - 1
                    if 0 < ni < nn[0] - 1 and 0 < nj < nn[1] - 1 and 0 < nk < nn[2] - 1:
                        direct[c, nk, nj, ni] += star[v, i]
    stored = np.zeros_like(direct)
    count = np.zeros(direct.shape, dtype=int)
    ncol = 3 * nv[0]

    def taps(m):
        return [(m >> 1, 2), ((m >> 1) + 1, 0)] if m & 1 else [(m >> 1, 1)]

    for cz in range(n[2]):
        for cy in range(n[1]):
            for cx in range(n[0]):
                for c in range(3):
                    for b2 in range(3):
                        for b1 in range(3):
                            nj, nk = 2 * cy + b1, 2 * cz + b2
                            u = np.zeros(3)
                            if 0 < nj < nn[1] - 1 and 0 < nk < nn[2] - 1:
                                acc = np.zeros(3)
                                for vz_, oz in taps(nk):
                                    for vy_, oy in taps(nj):
                                        row = ((c * 3 + oz) * 3 + oy) * (nv[1] * nv[2]) + vz_ * nv[1] + vy_
                                        rp = row * ncol + 3 * cx
                                        acc += [out[rp + 1], out[rp + 2] + out[rp + 3], out[rp + 4]]
                                for a in range(3):
                                    ni = 2 * cx + a
                                    u[a] = 0.0 if ni in (0, nn[0] - 1) else acc[a]
                            for a in range(3):
                                ni = 2 * cx + a
                                assert u[a] == pytest.approx(direct[c, nk, nj, ni], abs=1e-12)
                            if (b1 < 2 or cy == n[1] - 1) and (b2 < 2 or cz == n[2] - 1):
                                for a in range(3):
                                    if a < 2 or cx == n[0] - 1:
                                        stored[c, nk, nj, 2 * cx + a] = u[a]
                                        count[c, nk, nj, 2 * cx + a] += 1
    assert np.all(count == 1)
    assert np.allclose(stored, direct, atol=1e-12)


def _launch_batch_tables(blocks, kmax=64):
    """csrc/batch.cuh, launch_batch: consecutive groups of at most kmax items with blocks,
    each a table of start offsets (items with no blocks left out)."""
    tables, i = [], 0
    while i < len(blocks):
        start, items, total = [], [], 0
        while i < len(blocks) and len(items) < kmax:
            if blocks[i]:
                start.append(total)
                items.append(i)
                total += blocks[i]
            i += 1
        start.append(total)
        if items:
            tables.append((start, items))
    return tables


def _batch_slot(start, count, b):
    lo, hi = 0, count - 1
    while lo < hi:
        mid = (lo + hi + 1) >> 1
        if start[mid] <= b:
            lo = mid
        else:
            hi = mid - 1
    return lo


@pytest.mark.parametrize("seed", range(4))
def test_merged_launch_work_list(seed):
    """Merged batch launches (csrc/batch.cuh): every block of every launch finds, by the
    binary search over the start offsets, the one item whose range holds it, and each item
    with blocks gets exactly its blocks, once, with local indices 0 .. blocks - 1; items
    with none get no launch slot.  Persistent shares: at least one block and at most
    min(work, cap) per item with work, none without, in proportion to the work."""
    rng = np.random.default_rng(seed)
    n = int(rng.integers(1, 150))
    blocks = [int(b) for b in rng.integers(0, 9, n) * (rng.random(n) < 0.8)]
    seen = {}
    for start, items in _launch_batch_tables(blocks):
        assert len(items) <= 64
        for b in range(start[-1]):
            s = _batch_slot(start, len(items), b)
            assert start[s] <= b < start[s + 1]
            seen.setdefault(items[s], []).append(b - start[s])
    for i, nb in enumerate(blocks):
        assert sorted(seen.get(i, [])) == list(range(nb))
    work = [int(w) for w in rng.integers(0, 5000, n)]
    cap, capacity = int(rng.integers(1, 64)), int(rng.integers(100, 3000))
    W = sum(work)
    shares = []
    for w in work:
        b = 0 if w <= 0 else min(max(-(-capacity * w // W), 1), w, cap)
        shares.append(b)
        if w:
            assert 1 <= b <= min(w, cap)
        else:
            assert b == 0
    if W:
        assert sum(shares) <= capacity + n
