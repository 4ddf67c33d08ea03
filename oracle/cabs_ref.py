"""Plain FP64 CPU oracle for cascaded bilateral sampling (CABS), arXiv 1607.07395.

TEST INFRASTRUCTURE ONLY. This module is imported by ``tests/``, by
``__graft_entry__.smoke()`` and by the CPU-baseline leg of ``bench.py``; the
GPU library never imports, links or executes it, and the two share no code.
It is slow on purpose: every step is written the way the paper states it,
in FP64, with numpy's LAPACK SVD and plain array operations as the only
library primitives.

Steps and the passages they follow (section / equation / algorithm of the paper):

=====================  ===================================================
``philox4x64_10``      counter-based generator (Salmon et al., SC'11) used to
                       draw the random indices; the paper only says
                       "randomly select" (Algorithm 2, step 1)
``draw_indices``       k distinct uniform indices: partial Fisher-Yates over a
                       virtual identity array (Algorithm 2, step 1)
``gather_dense`` /     C = A[:, I^c], R = A[I^r, :] (kept transposed, n x k,
``gather_rbf``         as in the proof of Theorem 1), W = A[I^r, I^c]
                       (Algorithm 2, steps 1 and 3)
``sketching``          SVD of W, extrapolation C V_w and R^T U_w, column-norm
                       normalisation N_c, N_r, and the scale S: the stabilised
                       form (Section 4.1, unnumbered equation after Eq. W) or
                       the pseudo-skeleton C W^+ R (Section 2.2, Eq. W)
``embed``              P = U S^(1/2), Q = V S^(1/2) (Algorithm 2, step 2)
``weighted_kmeans``    Lloyd iterations minimising the weighted encoding error
                       (Section 3.2, Eq. wkmeans) from the pilot rows
``snap``               every centre replaced by its closest in-sample point
                       (Section 3.2, last paragraph)
``hard_threshold``     follow-up by the k2 largest-norm rows (Section 5,
                       follow-up variant (f))
``leverage_scores`` /  follow-up by approximate leverage scores (Section 5,
``weighted_sample``    variant (e)): squared row norms of the orthonormal
                       factors of the pilot sketch (supplementary Section 3
                       names leverage scores as the use of that form), used
                       as sampling probabilities without replacement
``CSRSource``          sparse A in compressed rows (Table 1's sparse inputs)
``cabs``               Algorithm 2 end to end
``orthogonalize``      the sketch in SVD form (supplementary Section 3)
``pinv_trunc``         pseudo-inverse by the SVD with the truncation below
``br_cur``             Bilateral Resampling CUR with given base and target
                       samplings (Section 2.2, Algorithm 1)
``sketch_cur``         Sketch-CUR: BR-CUR with independent random base and
                       target samplings, target three times the base
                       (Section 2.2 item 3; Section 5, comparison (a))
``rel_fro_error_*``    |A - U S V^T|_F / |A|_F (Section 5), exact or on
                       uniformly sampled entries
=====================  ===================================================

Readings where the paper is silent (the GPU library takes the same ones):

* Index draw: Philox4x64-10 with key (seed, tag), tag 0 = rows, 1 = columns,
  2 = error-estimate samples, 4 / 5 = Sketch-CUR target rows / columns,
  6 / 7 = leverage-score follow-up rows / columns; counter (i, 0, 0, 0) for the i-th draw; output
  word 0 mapped to [0, N - i) by the high half of the 128-bit product
  (multiply-shift, bias <= N / 2^64). The drawn indices are returned in draw
  order and sorted ascending; W, C and R use the sorted order.
* Truncation: singular values sigma_i <= max(trunc_rtol, k * 2^-52) * sigma_1
  are dropped (k * eps * sigma_1 is MATLAB ``pinv``'s default tolerance; the
  paper ran MATLAB). Dropped components give zero columns in U, V and zero S.
  A component whose extrapolated norm is zero is dropped the same way.
* Stabilised scale: S = Sigma_w * sqrt(m n / (k_r k_c)) (k_r = k_c = k in the
  paper's equation).
* k-means: init = P at the first k2 pilot rows in draw order; exactly ``iters``
  rounds of {assign, update}; squared distances by direct differences; ties go
  to the lowest centre index; weights Upsilon(t) = t^p with 0^0 = 1; an empty
  cluster (zero total weight) keeps its centre.
* Snap: centres processed in index order, each taking the nearest row not yet
  taken; ties go to the lowest row index, a tie meaning a squared distance
  within 1e-12 (d* + |z|^2) of the nearest d* (the centre of a two-row
  cluster is equidistant from both rows, and rounding alone would otherwise
  pick one); the result is then sorted.

Every function here is pinned by tests in ``tests/test_oracle_*.py`` against
facts the paper or mathematics fixes (numpy's independent Philox, closed-form
recoveries, brute force on tiny inputs, invariants). No function is left
unpinned.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

TAG_ROWS = 0
TAG_COLS = 1
TAG_EVAL = 2
TAG_TARGET_ROWS = 4
TAG_TARGET_COLS = 5
TAG_LEV_ROWS = 6
TAG_LEV_COLS = 7

MASK64 = (1 << 64) - 1
_M0 = 0xD2E7470EE14C6C93
_M1 = 0xCA5A826395121157
_W0 = 0x9E3779B97F4A7C15
_W1 = 0xBB67AE8584CAA73B
EPS64 = 2.0 ** -52


# --------------------------------------------------------------------------
# Counter-based random numbers (Philox4x64-10, Salmon et al. 2011)
# --------------------------------------------------------------------------

def philox4x64_10(counter, key):
    """One Philox4x64-10 block: 10 rounds of two 64x64->128 multiplies, with the
    key bumped by the Weyl constants between rounds. Plain Python integers."""
    c0, c1, c2, c3 = (int(x) & MASK64 for x in counter)
    k0, k1 = (int(x) & MASK64 for x in key)
    for _ in range(10):
        p0 = _M0 * c0
        p1 = _M1 * c2
        c0, c1, c2, c3 = ((p1 >> 64) ^ c1 ^ k0, p1 & MASK64, (p0 >> 64) ^ c3 ^ k1, p0 & MASK64)
        k0 = (k0 + _W0) & MASK64
        k1 = (k1 + _W1) & MASK64
    return c0, c1, c2, c3


def mulhi64(a: int, b: int) -> int:
    """High 64 bits of the 128-bit product a * b."""
    return ((int(a) & MASK64) * (int(b) & MASK64)) >> 64


def _mulhilo_u64(a: np.ndarray, b: np.ndarray):
    """Vectorised 64x64->128 multiply of uint64 arrays via 32-bit halves."""
    m32 = np.uint64(0xFFFFFFFF)
    s32 = np.uint64(32)
    a_lo, a_hi = a & m32, a >> s32
    b_lo, b_hi = b & m32, b >> s32
    p0 = a_lo * b_lo
    p1 = a_lo * b_hi
    p2 = a_hi * b_lo
    p3 = a_hi * b_hi
    mid = (p0 >> s32) + (p1 & m32) + (p2 & m32)
    hi = p3 + (p1 >> s32) + (p2 >> s32) + (mid >> s32)
    lo = a * b
    return hi, lo


def philox4x64_10_vec(c0, c1, c2, c3, k0: int, k1: int):
    """Philox4x64-10 on arrays of counters (same key); returns four uint64 arrays."""
    c0, c1, c2, c3 = (np.asarray(x, dtype=np.uint64).copy() for x in (c0, c1, c2, c3))
    k0 = np.uint64(k0 & MASK64)
    k1 = np.uint64(k1 & MASK64)
    m0, m1 = np.uint64(_M0), np.uint64(_M1)
    w0, w1 = np.uint64(_W0), np.uint64(_W1)
    with np.errstate(over="ignore"):
        for _ in range(10):
            hi0, lo0 = _mulhilo_u64(np.full_like(c0, m0), c0)
            hi1, lo1 = _mulhilo_u64(np.full_like(c2, m1), c2)
            c0, c1, c2, c3 = hi1 ^ c1 ^ k0, lo1, hi0 ^ c3 ^ k1, lo0
            k0 = k0 + w0
            k1 = k1 + w1
    return c0, c1, c2, c3


def mulhi64_vec(a: np.ndarray, n) -> np.ndarray:
    """High 64 bits of a * n for a uint64 array a and scalar/array n."""
    hi, _ = _mulhilo_u64(np.asarray(a, dtype=np.uint64), np.asarray(n, dtype=np.uint64) + np.zeros_like(a))
    return hi


# --------------------------------------------------------------------------
# Algorithm 2, step 1: pilot sampling of k rows and k columns
# --------------------------------------------------------------------------

def draw_indices(seed: int, tag: int, N: int, k: int):
    """k distinct uniform indices from [0, N): partial Fisher-Yates.

    Step i swaps position i of a virtual identity array with position
    j = i + floor(r_i (N - i) / 2^64), r_i = word 0 of Philox((i,0,0,0), (seed, tag)).
    The array is held as a sparse map of the positions that were touched.
    Returns (indices in draw order, indices sorted ascending), both int64."""
    if not (0 <= k <= N):
        raise ValueError("need 0 <= k <= N")
    moved = {}
    drawn = []
    for i in range(k):
        r = philox4x64_10((i, 0, 0, 0), (seed, tag))[0]
        j = i + mulhi64(r, N - i)
        vi = moved.get(i, i)
        vj = moved.get(j, j)
        moved[j] = vi
        moved[i] = vj
        drawn.append(vj)
    drawn = np.array(drawn, dtype=np.int64)
    return drawn, np.sort(drawn)


# --------------------------------------------------------------------------
# Algorithm 2, steps 1 and 3: gathers
# --------------------------------------------------------------------------

def gather_dense(A: np.ndarray, rows, cols):
    """C = A[:, cols] (m x k_c), R^T = A[rows, :]^T (n x k_r), W = A[rows, cols] (k_r x k_c).

    Values are widened to FP64 (exact from FP32)."""
    rows = np.asarray(rows)
    cols = np.asarray(cols)
    C = np.array(A[:, cols], dtype=np.float64)
    Rt = np.array(A[rows, :].T, dtype=np.float64)
    W = np.array(A[np.ix_(rows, cols)], dtype=np.float64)
    return C, Rt, W


def rbf_entries(X: np.ndarray, Y: np.ndarray, sigma: float, ii, jj) -> np.ndarray:
    """Entries exp(-|x_i - y_j|^2 / (2 sigma^2)) for paired index arrays, in FP64."""
    x = np.asarray(X, dtype=np.float64)[np.asarray(ii)]
    y = np.asarray(Y, dtype=np.float64)[np.asarray(jj)]
    s = float(sigma)
    d2 = ((x - y) ** 2).sum(axis=-1)
    return np.exp(-d2 / (2.0 * s * s))


def rbf_block(X, Y, sigma, rows, cols) -> np.ndarray:
    """The block A[rows, cols] of the implicit RBF matrix in FP64."""
    x = np.asarray(X, dtype=np.float64)[np.asarray(rows)]
    y = np.asarray(Y, dtype=np.float64)[np.asarray(cols)]
    s = float(sigma)
    out = np.empty((x.shape[0], y.shape[0]))
    for t in range(y.shape[0]):
        out[:, t] = np.exp(-((x - y[t]) ** 2).sum(axis=1) / (2.0 * s * s))
    return out


def gather_rbf(X, Y, sigma, rows, cols):
    """C, R^T, W of the implicit RBF matrix, generated in FP64 from the FP32 points."""
    m, n = X.shape[0], Y.shape[0]
    C = rbf_block(X, Y, sigma, np.arange(m), cols)
    Rt = rbf_block(X, Y, sigma, rows, np.arange(n)).T.copy()
    W = rbf_block(X, Y, sigma, rows, cols)
    return C, Rt, W


# --------------------------------------------------------------------------
# Section 4.1: the sketching routine
# --------------------------------------------------------------------------

@dataclass
class Sketch:
    U: np.ndarray          # m x k, zero columns beyond the kept components
    S: np.ndarray          # k
    V: np.ndarray          # n x k
    rank: int              # number of kept singular values of W
    Uw: np.ndarray = None
    sig: np.ndarray = None
    Vw: np.ndarray = None
    Nc: np.ndarray = None
    Nr: np.ndarray = None


def sketching(C: np.ndarray, Rt: np.ndarray, W: np.ndarray, m: int, n: int,
              mode: str = "pinv", trunc_rtol: float = 0.0) -> Sketch:
    """Decomposition A ~ U diag(S) V^T from sampled columns C, rows R (given as
    R^T) and their intersection W.

    SVD W = U_w Sigma_w V_w^T (Section 4.1). The right singular vectors are
    extrapolated through the columns, C V_w, and the left ones through the
    rows, R^T U_w; N_c and N_r are their column norms; U = C V_w N_c^-1 and
    V = R^T U_w N_r^-1 (n x k, the transpose of the paper's N_r^-1 U_w^T R).

    mode "stabilized": S = Sigma_w sqrt(m n) / k (the stabilised form).
    mode "pinv":       S = N_c N_r Sigma_w^-1, which makes U S V^T = C W^+ R,
                       the pseudo-skeleton approximation (Section 2.2, Eq. W).
    """
    k_r, k_c = W.shape
    k = max(k_r, k_c)
    Uw, sig, Vwt = np.linalg.svd(W)
    Vw = Vwt.T
    ncomp = min(k_r, k_c)
    if sig.size == 0 or sig[0] <= 0.0:
        r = 0
    else:
        tol = max(trunc_rtol, k * EPS64) * sig[0]
        r = int(np.count_nonzero(sig > tol))
    a = C @ Vw[:, :r]
    b = Rt @ Uw[:, :r]
    Nc = np.sqrt((a * a).sum(axis=0))
    Nr = np.sqrt((b * b).sum(axis=0))
    ok = (Nc > 0) & (Nr > 0)
    U = np.zeros((C.shape[0], ncomp))
    V = np.zeros((Rt.shape[0], ncomp))
    S = np.zeros(ncomp)
    for i in range(r):
        if not ok[i]:
            continue
        U[:, i] = a[:, i] / Nc[i]
        V[:, i] = b[:, i] / Nr[i]
        if mode == "stabilized":
            S[i] = sig[i] * math.sqrt(m * n / (k_r * k_c))
        elif mode == "pinv":
            S[i] = Nc[i] * Nr[i] / sig[i]
        else:
            raise ValueError(mode)
    return Sketch(U=U, S=S, V=V, rank=r, Uw=Uw, sig=sig, Vw=Vw, Nc=Nc, Nr=Nr)


def embed(U: np.ndarray, S: np.ndarray) -> np.ndarray:
    """Low-rank embedding P = U S^(1/2) (Algorithm 2, step 2)."""
    return U * np.sqrt(S)[None, :]


# --------------------------------------------------------------------------
# Section 3.2: weighted k-means sampling and snapping
# --------------------------------------------------------------------------

def upsilon_weights(X: np.ndarray, p: float) -> np.ndarray:
    """Row weights Upsilon(|X_l|_2) with the power function Upsilon(t) = t^p (0^0 = 1)."""
    nrm = np.sqrt((X * X).sum(axis=1))
    if p == 0.0:
        return np.ones(X.shape[0])
    return nrm ** p


def sq_dists_to(X: np.ndarray, z: np.ndarray) -> np.ndarray:
    """Squared Euclidean distances of every row of X to the point z, by direct differences."""
    d = X - z[None, :]
    return (d * d).sum(axis=1)


@dataclass
class KMeansResult:
    labels: list = field(default_factory=list)     # per iteration, int64 (M,)
    energy: list = field(default_factory=list)     # weighted encoding error per iteration
    margin: list = field(default_factory=list)     # (second best - best) per iteration
    best: list = field(default_factory=list)       # best squared distance per iteration
    centres: list = field(default_factory=list)    # centres used by each iteration, then the final ones
    weights: np.ndarray = None

    @property
    def Z(self) -> np.ndarray:
        return self.centres[-1]


def weighted_kmeans(X: np.ndarray, init_rows, iters: int, upsilon_pow: float = 0.0) -> KMeansResult:
    """Lloyd iterations on the weighted objective sum_l w_l |X_l - Z_s(l)|^2
    (Eq. wkmeans), w_l = Upsilon(|X_l|), starting from Z = X[init_rows]."""
    X = np.asarray(X, dtype=np.float64)
    M = X.shape[0]
    Z = X[np.asarray(init_rows)].copy()
    k2 = Z.shape[0]
    w = upsilon_weights(X, upsilon_pow)
    res = KMeansResult(weights=w)
    for _ in range(iters):
        res.centres.append(Z.copy())
        D = np.empty((M, k2))
        for j in range(k2):
            D[:, j] = sq_dists_to(X, Z[j])
        s = np.argmin(D, axis=1)
        best = D[np.arange(M), s]
        if k2 > 1:
            D2 = D.copy()
            D2[np.arange(M), s] = np.inf
            margin = D2.min(axis=1) - best
        else:
            margin = np.full(M, np.inf)
        res.labels.append(s)
        res.best.append(best)
        res.margin.append(margin)
        res.energy.append(float((w * best).sum()))
        Znew = Z.copy()
        for j in range(k2):
            mem = s == j
            wsum = w[mem].sum()
            if wsum > 0:
                Znew[j] = (w[mem, None] * X[mem]).sum(axis=0) / wsum
        Z = Znew
    res.centres.append(Z.copy())
    return res


def encoding_error(X: np.ndarray, reps_rows, upsilon_pow: float = 0.0):
    """Weighted encoding error of X with representatives X[reps_rows] and the
    nearest-representative assignment (Eq. eer / Eq. wkmeans). Returns
    (error, labels, max cluster size T of Eq. T)."""
    X = np.asarray(X, dtype=np.float64)
    Z = X[np.asarray(reps_rows)]
    D = np.empty((X.shape[0], Z.shape[0]))
    for j in range(Z.shape[0]):
        D[:, j] = sq_dists_to(X, Z[j])
    s = np.argmin(D, axis=1)
    w = upsilon_weights(X, upsilon_pow)
    err = float((w * D[np.arange(X.shape[0]), s]).sum())
    T = int(np.bincount(s, minlength=Z.shape[0]).max()) if X.shape[0] else 0
    return err, s, T


SNAP_TIE_RTOL = 1e-12


def snap(X: np.ndarray, Z: np.ndarray, tie_rtol: float = SNAP_TIE_RTOL):
    """Replace each centre by its closest in-sample row of X, all distinct.

    Centres are taken in index order; each takes the nearest row not already
    taken. Ties go to the lowest row index, where a tie is judged at the
    resolution of the arithmetic: with d* the smallest squared distance of an
    untaken row to the centre z, every untaken row with
    d <= d* + tie_rtol (d* + |z|^2) is tied with the nearest. Exact ties are
    structural here, not accidental: the centre of a cluster of two rows of
    equal weight is their midpoint, equidistant from both, and which of the
    two rounded distances comes out smaller depends only on the order of the
    floating-point sum. Returns (rows in centre order, sorted rows)."""
    X = np.asarray(X, dtype=np.float64)
    taken = np.zeros(X.shape[0], dtype=bool)
    out = []
    for j in range(Z.shape[0]):
        z = np.asarray(Z[j], dtype=np.float64)
        d = sq_dists_to(X, z)
        d[taken] = np.inf
        dstar = d.min()
        l = int(np.flatnonzero(d <= dstar + tie_rtol * (dstar + float((z * z).sum())))[0])
        taken[l] = True
        out.append(l)
    out = np.array(out, dtype=np.int64)
    return out, np.sort(out)


def leverage_scores(X: np.ndarray) -> np.ndarray:
    """Leverage scores of the rows of an orthonormal basis X: |X_i|^2."""
    X = np.asarray(X, dtype=np.float64)
    return (X * X).sum(axis=1)


def philox_uniform(seed: int, tag: int, N: int) -> np.ndarray:
    """u_i = ((r_i >> 11) + 1/2) 2^-53 in (0, 1), r_i = word 0 of
    Philox((i, 0, 0, 0), (seed, tag)), i = 0..N-1 (exact in FP64)."""
    c0 = np.arange(N, dtype=np.uint64)
    z = np.zeros(N, dtype=np.uint64)
    r0 = philox4x64_10_vec(c0, z, z, z, seed, tag)[0]
    return ((r0 >> np.uint64(11)).astype(np.float64) + 0.5) * 2.0 ** -53


def weighted_sample(w: np.ndarray, k: int, seed: int, tag: int):
    """k distinct indices drawn without replacement with probabilities
    proportional to w (the A-Res scheme of Efraimidis and Spirakis, 2006):
    index i gets the key u_i^(1/w_i), u_i = philox_uniform(seed, tag)_i, and
    the k largest keys win. The keys are ranked through the increasing map
    u^(1/w) -> w / (-ln u), evaluated in FP64; ties go to the lower index, and
    w_i = 0 gives key 0. Returns (selected indices ascending, keys)."""
    w = np.asarray(w, dtype=np.float64)
    N = len(w)
    if not (0 <= k <= N):
        raise ValueError("need 0 <= k <= N")
    u = philox_uniform(seed, tag, N)
    keys = w / -np.log(u)
    order = np.lexsort((np.arange(N), -keys))
    return np.sort(order[:k]), keys


def hard_threshold(X: np.ndarray, k2: int):
    """Follow-up selection by hard threshold (Section 5, follow-up variant (f)):
    instead of clustering, keep the k2 rows whose weight Upsilon(|X_l|_2) is
    largest. Upsilon is monotone, so this ranks rows by the embedding norm
    itself (for a constant Upsilon every weight ties; ranking by the norm is
    the limit of any increasing Upsilon). Squared norms are summed in FP64 in
    dimension order; ties go to the lower row index. Returns the rows sorted."""
    X = np.asarray(X, dtype=np.float64)
    M = X.shape[0]
    if not (1 <= k2 <= M):
        raise ValueError("need 1 <= k2 <= M")
    sq = np.zeros(M)
    for q in range(X.shape[1]):
        sq = sq + X[:, q] * X[:, q]
    order = np.lexsort((np.arange(M), -sq))  # largest norm first, then lowest index
    return np.sort(order[:k2]).astype(np.int64)


# --------------------------------------------------------------------------
# Algorithm 2 end to end
# --------------------------------------------------------------------------

class DenseSource:
    """A stored matrix A (m x n)."""

    def __init__(self, A):
        self.A = A
        self.m, self.n = A.shape

    def gather(self, rows, cols):
        return gather_dense(self.A, rows, cols)

    def entries(self, ii, jj):
        return np.asarray(self.A[np.asarray(ii), np.asarray(jj)], dtype=np.float64)


class RBFSource:
    """The implicit RBF kernel matrix exp(-|x_i - y_j|^2 / 2 sigma^2)."""

    def __init__(self, X, Y, sigma):
        self.X, self.Y, self.sigma = X, Y, float(sigma)
        self.m, self.n = X.shape[0], Y.shape[0]

    def gather(self, rows, cols):
        return gather_rbf(self.X, self.Y, self.sigma, rows, cols)

    def entries(self, ii, jj):
        return rbf_entries(self.X, self.Y, self.sigma, ii, jj)


class CSRSource:
    """A sparse A (the sparse inputs of Table 1) in compressed rows: indptr
    (m + 1), indices (sorted within each row), data; missing entries are 0.
    Gathers go through scipy's sparse slicing, an implementation independent
    of the dense one."""

    def __init__(self, indptr, indices, data, n):
        import scipy.sparse as sp
        indptr = np.asarray(indptr)
        self.m, self.n = len(indptr) - 1, int(n)
        self.A = sp.csr_matrix((np.asarray(data), np.asarray(indices), indptr), shape=(self.m, self.n))

    def gather(self, rows, cols):
        rows = np.asarray(rows)
        cols = np.asarray(cols)
        C = np.asarray(self.A[:, cols].toarray(), dtype=np.float64)
        Rt = np.asarray(self.A[rows, :].toarray().T, dtype=np.float64)
        W = np.asarray(self.A[rows, :][:, cols].toarray(), dtype=np.float64)
        return C, Rt, W

    def entries(self, ii, jj):
        return np.asarray(self.A[np.asarray(ii), np.asarray(jj)], dtype=np.float64).ravel()

    def dense(self):
        return np.asarray(self.A.toarray(), dtype=np.float64)


@dataclass
class CabsResult:
    pilot_rows: np.ndarray
    pilot_cols: np.ndarray
    pilot_rows_drawn: np.ndarray
    pilot_cols_drawn: np.ndarray
    pilot: Sketch
    P: np.ndarray
    Q: np.ndarray
    km_rows: KMeansResult
    km_cols: KMeansResult
    rows: np.ndarray            # follow-up row indices, sorted
    cols: np.ndarray            # follow-up column indices, sorted
    rows_centre_order: np.ndarray
    cols_centre_order: np.ndarray
    final: Sketch
    e_pilot: tuple = None       # (e^r_p, e^c_p)
    e_follow: tuple = None      # (e^r_f, e^c_f)
    T_pilot: tuple = None
    T_follow: tuple = None


def cabs(source, k1: int, k2: int = None, iters: int = 5, seed: int = 1607,
         mode: str = "pinv", upsilon_pow: float = 0.0, trunc_rtol: float = 0.0,
         follow: str = "kmeans") -> CabsResult:
    """Cascaded bilateral sampling (Algorithm 2).

    1. pilot sampling of k1 random rows and columns; 2. pilot sketching and
    embeddings P, Q; 3. weighted k-means on P and on Q, centres snapped to
    rows -> follow-up indices (follow="threshold" or "leverage": the
    hard-threshold or leverage-score variant of Section 5 instead);
    4. follow-up sketching on the new gather."""
    k2 = k1 if k2 is None else k2
    m, n = source.m, source.n
    if not (1 <= k2 <= k1 <= min(m, n)):
        raise ValueError("need 1 <= k2 <= k1 <= min(m, n)")
    Ir_drawn, Ir = draw_indices(seed, TAG_ROWS, m, k1)
    Ic_drawn, Ic = draw_indices(seed, TAG_COLS, n, k1)
    C, Rt, W = source.gather(Ir, Ic)
    pilot = sketching(C, Rt, W, m, n, mode, trunc_rtol)
    P = embed(pilot.U, pilot.S)
    Q = embed(pilot.V, pilot.S)
    if follow == "threshold":
        km_r = km_c = None
        rows_o = rows = hard_threshold(P, k2)
        cols_o = cols = hard_threshold(Q, k2)
    elif follow == "leverage":
        # Section 5 variant (e): the pilot sketch P Q^T in SVD form
        # (supplementary Section 3), its leverage scores as probabilities
        km_r = km_c = None
        X, _, Y = orthogonalize(P, np.ones(k1), Q, trunc_rtol)
        rows_o = rows = weighted_sample(leverage_scores(X), k2, seed, TAG_LEV_ROWS)[0]
        cols_o = cols = weighted_sample(leverage_scores(Y), k2, seed, TAG_LEV_COLS)[0]
    elif follow == "kmeans":
        km_r = weighted_kmeans(P, Ir_drawn[:k2], iters, upsilon_pow)
        km_c = weighted_kmeans(Q, Ic_drawn[:k2], iters, upsilon_pow)
        rows_o, rows = snap(P, km_r.Z)
        cols_o, cols = snap(Q, km_c.Z)
    else:
        raise ValueError("follow must be 'kmeans', 'threshold' or 'leverage'")
    Cb, Rtb, Wb = source.gather(rows, cols)
    final = sketching(Cb, Rtb, Wb, m, n, mode, trunc_rtol)
    ep_r, _, Tp_r = encoding_error(P, Ir_drawn[:k2], upsilon_pow)
    ep_c, _, Tp_c = encoding_error(Q, Ic_drawn[:k2], upsilon_pow)
    ef_r, _, Tf_r = encoding_error(P, rows, upsilon_pow)
    ef_c, _, Tf_c = encoding_error(Q, cols, upsilon_pow)
    return CabsResult(pilot_rows=Ir, pilot_cols=Ic, pilot_rows_drawn=Ir_drawn,
                      pilot_cols_drawn=Ic_drawn, pilot=pilot, P=P, Q=Q, km_rows=km_r,
                      km_cols=km_c, rows=rows, cols=cols, rows_centre_order=rows_o,
                      cols_centre_order=cols_o, final=final, e_pilot=(ep_r, ep_c),
                      e_follow=(ef_r, ef_c), T_pilot=(Tp_r, Tp_c), T_follow=(Tf_r, Tf_c))


# --------------------------------------------------------------------------
# Supplementary Section 3: orthogonalisation of the sketch
# --------------------------------------------------------------------------

def orthogonalize(U: np.ndarray, S: np.ndarray, V: np.ndarray, trunc_rtol: float = 0.0):
    """The sketch U diag(S) V^T (U m x r, V n x r, S r) rewritten in SVD form
    with orthonormal factors, in O((m + n) r^2) (supplementary Section 3):
    the thin SVD U = U_0 Sigma_0 V_0^T, then the SVD of the r x n matrix
    Sigma_0 V_0^T diag(S) V^T = U_1 Sigma_1 V_1^T, giving
    A ~ (U_0 U_1) Sigma_1 V_1^T. Components with
    Sigma_1,i <= max(trunc_rtol, r 2^-52) Sigma_1,1 are dropped.
    Returns (U_0 U_1, diag(Sigma_1), V_1)."""
    U = np.asarray(U, dtype=np.float64)
    V = np.asarray(V, dtype=np.float64)
    S = np.asarray(S, dtype=np.float64)
    U0, s0, V0t = np.linalg.svd(U, full_matrices=False)
    B = (s0[:, None] * V0t) @ (S[:, None] * V.T)
    U1, s1, V1t = np.linalg.svd(B, full_matrices=False)
    r = len(s1)
    keep = s1 > max(trunc_rtol, r * 2.0 ** -52) * (s1[0] if r else 0.0)
    return U0 @ U1[:, keep], s1[keep], V1t.T[:, keep]


# --------------------------------------------------------------------------
# Section 2.2, Algorithm 1: BR-CUR and Sketch-CUR
# --------------------------------------------------------------------------

def pinv_trunc(B: np.ndarray, trunc_rtol: float = 0.0) -> np.ndarray:
    """Pseudo-inverse V diag(1/s) U^T of B = U diag(s) V^T over the singular
    values s_i > max(trunc_rtol, kmax 2^-52) s_1, kmax = max(B.shape).
    Algorithm 1 leaves the tolerance open; the floor is MATLAB pinv's default
    (the paper ran MATLAB, Section 5), the floor of the sketching routine
    too. Data that carry less than FP64 precision pass their resolution in
    trunc_rtol, as for the sketching routine."""
    B = np.asarray(B, dtype=np.float64)
    Ub, sb, Vbt = np.linalg.svd(B, full_matrices=False)
    if len(sb) == 0 or sb[0] == 0.0:
        return np.zeros(B.T.shape)
    keep = sb > max(trunc_rtol, max(B.shape) * EPS64) * sb[0]
    return (Vbt[keep].T / sb[keep]) @ Ub[:, keep].T


@dataclass
class CurResult:
    rows_b: np.ndarray   # base rows I^b_r, sorted
    cols_b: np.ndarray   # base columns I^b_c, sorted
    rows_t: np.ndarray   # target rows I^t_r, sorted
    cols_t: np.ndarray   # target columns I^t_c, sorted
    C: np.ndarray        # m x k_b
    U: np.ndarray        # k_b x k_b, U*
    Rt: np.ndarray       # n x k_b, R^T


def br_cur(source, rows_b, cols_b, rows_t, cols_t, trunc_rtol: float = 0.0) -> CurResult:
    """Algorithm 1 with the given samplings: bases C = A[:, I^b_c] and
    R = A[I^b_r, :] (step 1), their samples C_bar = C[I^t_r, :] and
    R_bar = R[:, I^t_c] (step 2), the target block M = A[I^t_r, I^t_c]
    (step 3), U* = C_bar^+ M R_bar^+, the minimiser of |M - C_bar U R_bar|_F
    (step 4); A ~ C U* R (step 5)."""
    rows_b, cols_b = np.asarray(rows_b), np.asarray(cols_b)
    rows_t, cols_t = np.asarray(rows_t), np.asarray(cols_t)
    C, Rt, _ = source.gather(rows_b, cols_b)
    Cbar = C[rows_t, :]
    Rbar = Rt[cols_t, :].T
    _, _, M = source.gather(rows_t, cols_t)
    Ustar = pinv_trunc(Cbar, trunc_rtol) @ M @ pinv_trunc(Rbar, trunc_rtol)
    return CurResult(rows_b=rows_b, cols_b=cols_b, rows_t=rows_t, cols_t=cols_t, C=C, U=Ustar, Rt=Rt)


def sketch_cur(source, kb: int, kt: int = None, seed: int = 1607, trunc_rtol: float = 0.0) -> CurResult:
    """Sketch-CUR: BR-CUR with independent uniform base (k_b rows and
    columns, tags 0 and 1, as the pilot draw of Algorithm 2) and target
    (k_t = 3 k_b by default, tags 4 and 5) samplings."""
    kt = 3 * kb if kt is None else kt
    m, n = source.m, source.n
    if not (1 <= kb <= min(m, n) and 1 <= kt <= min(m, n)):
        raise ValueError("need 1 <= kb, kt <= min(m, n)")
    _, rows_b = draw_indices(seed, TAG_ROWS, m, kb)
    _, cols_b = draw_indices(seed, TAG_COLS, n, kb)
    _, rows_t = draw_indices(seed, TAG_TARGET_ROWS, m, kt)
    _, cols_t = draw_indices(seed, TAG_TARGET_COLS, n, kt)
    return br_cur(source, rows_b, cols_b, rows_t, cols_t, trunc_rtol)


# --------------------------------------------------------------------------
# Section 5: relative Frobenius error
# --------------------------------------------------------------------------

def rel_fro_error_dense(A: np.ndarray, U: np.ndarray, S: np.ndarray, V: np.ndarray,
                        row_block: int = 512) -> float:
    """|A - U diag(S) V^T|_F / |A|_F, exactly in FP64, one row block at a time."""
    num = 0.0
    den = 0.0
    US = np.asarray(U, dtype=np.float64) * np.asarray(S, dtype=np.float64)[None, :]
    V = np.asarray(V, dtype=np.float64)
    for r0 in range(0, A.shape[0], row_block):
        a = np.asarray(A[r0:r0 + row_block], dtype=np.float64)
        d = a - US[r0:r0 + row_block] @ V.T
        num += float((d * d).sum())
        den += float((a * a).sum())
    return math.sqrt(num / den) if den > 0 else 0.0


def eval_samples(seed: int, m: int, n: int, count: int):
    """Uniform (i, j) pairs with replacement for the sampled error: word 0 and
    word 1 of Philox((t,0,0,0), (seed, TAG_EVAL)) scaled to [0, m) and [0, n)."""
    t = np.arange(count, dtype=np.uint64)
    z = np.zeros_like(t)
    w0, w1, _, _ = philox4x64_10_vec(t, z, z, z, seed, TAG_EVAL)
    return mulhi64_vec(w0, m).astype(np.int64), mulhi64_vec(w1, n).astype(np.int64)


def rel_fro_error_sampled(source, U, S, V, seed: int, count: int) -> float:
    """sqrt(sum (a - a_hat)^2 / sum a^2) over ``count`` uniformly sampled entries."""
    ii, jj = eval_samples(seed, source.m, source.n, count)
    a = source.entries(ii, jj)
    US = np.asarray(U, dtype=np.float64) * np.asarray(S, dtype=np.float64)[None, :]
    ahat = (US[ii] * np.asarray(V, dtype=np.float64)[jj]).sum(axis=1)
    num = float(((a - ahat) ** 2).sum())
    den = float((a * a).sum())
    return math.sqrt(num / den) if den > 0 else 0.0
