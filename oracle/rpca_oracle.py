"""FP64 CPU oracle: the randomized block-Lanczos PCA of Section 3, step by step.

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).  Plain, slow and written
to be checked against the paper by eye: no blocking, fusion or reordering
beyond what the paper itself states.  Streaming of A by row blocks follows
Section 4.2 ("retrieve as many rows of A as fit in memory ...").

Steps (Section 3, eqs. first_prod .. product33):
  1. G n x l standard Gaussian;  H^(0) = A G;  H^(j) = A (A^T H^(j-1)),
     j = 1..i;  H = [H^(0) | ... | H^(i)]            (m x (i+1)l)
  2. pivoted QR:  H = Q R   (Q m x (i+1)l, orthonormal columns)
  3. T = A^T Q                                         (n x (i+1)l)
  4. SVD  T = V~ Sigma~ W^T, singular values descending
  5. U~ = Q W
  6. U = U~[:, :k],  V = V~[:, :k],  Sigma = Sigma~[:k, :k]
Section 3 assumes n <= m and applies the method to A^T otherwise.
Section 1 describes "normalizing" A by subtracting from each column its mean;
``center=True`` does exactly that on every row block (A_c = A - 1 c^T with
c the FP64 column means).

``normalize=True`` is the reading of the Remark on over/underflow at the end
of Section 3 (process a normalised iterate): after each F = A^T H^(j) the
oracle replaces F by the Q factor of its thin QR (positive diagonal R), so
H^(j+1) = A orth(F).  span(H) is unchanged in exact arithmetic.  The default
(raw) form is the paper's literal one.

``reorth=True`` (implies normalize) also takes out of F its components along
every earlier n-side block before orthonormalising it (block Gram-Schmidt,
applied twice), starting from X^(0) = orth(G): the block Lanczos form of the
same Krylov space.  span(X^(0..j)) is K_j = span(G, A^T A G, ...,
(A^T A)^j G) either way (K_{j+1} = K_j + A^T A X^(j)), so span(H) =
A K_i is unchanged; but H = A [X^(0) .. X^(i)] with orthonormal
[X^(0) .. X^(i)] has the condition number of A restricted to K_i, where the
normalised blocks alone give the condition of a Krylov basis (measured:
2e3 against 6 on the precision workload, 5e10 against 3e4 on the centred
one).  This is the form the GPU path computes.
"""
import numpy as np

from . import philox


class ParameterError(ValueError):
    pass


def check_parameters(m, n, k, l, i):
    """Parameter rules of Sections 2 and 3: 1 <= k < min(m, n), l >= k,
    i >= 0, and (i+1)l columns must fit: (i+1)l <= min(m, n).  (Section 3
    recommends (i+1)l <= n - k; exceeding that only weakens the bound, so it
    is not an error here.)"""
    if m < 1 or n < 1:
        raise ParameterError("empty matrix")
    if not (1 <= k < min(m, n)):
        raise ParameterError("need 1 <= k < min(m, n)")
    if l < k:
        raise ParameterError("need l >= k")
    if i < 0:
        raise ParameterError("need i >= 0")
    if (i + 1) * l > min(m, n):
        raise ParameterError("need (i+1) l <= min(m, n)")


# ----------------------------------------------------------------------------
# Row-block access to A (Section 4.2) with optional column centering (Sec. 1)
# ----------------------------------------------------------------------------
class RowSource:
    """Rows of an m x n matrix in FP64, delivered block by block.

    ``A`` is an ndarray (any real dtype; values are upcast exactly to FP64)
    or a callable ``rows(r0, r1) -> ndarray`` generating rows on the fly
    (Section 4.1).  ``col_scale`` (length n) multiplies column j by
    col_scale[j] after upcasting (stored low-precision values times their
    per-column scale)."""

    def __init__(self, A, m=None, n=None, block_rows=8192, col_scale=None):
        if callable(A):
            if m is None or n is None:
                raise ValueError("callable source needs m, n")
            self._rows, self.m, self.n = A, int(m), int(n)
        else:
            A = np.asarray(A)
            self.m, self.n = A.shape
            self._rows = lambda r0, r1: A[r0:r1]
        self.block_rows = int(block_rows)
        self.col_scale = None if col_scale is None else np.asarray(col_scale, np.float64)
        self.shift = None                       # column means when centering

    def blocks(self):
        for r0 in range(0, self.m, self.block_rows):
            r1 = min(self.m, r0 + self.block_rows)
            B = np.asarray(self._rows(r0, r1), dtype=np.float64)
            if self.col_scale is not None:
                B = B * self.col_scale[None, :]
            if self.shift is not None:
                B = B - self.shift[None, :]     # A_c = A - 1 c^T, materialised
            yield r0, r1, B

    def column_means(self):
        """c = (1/m) sum_i A_i (Section 1's column means), by the corrected
        two-pass algorithm (Chan, Golub and LeVeque, "Algorithms for
        computing the sample variance", 1983): a first pass gives c0, a
        second adds the mean of the residuals A_i - c0.  The residuals are
        small where the columns carry a large offset, so c is the mean to
        about one rounding of c itself; a plain sum of offset entries errs
        by ~u log(m) |c|, which on a centred workload shifts the data by a
        rank-one term large enough to move U."""
        saved, self.shift = self.shift, None
        s = np.zeros(self.n)
        for _, _, B in self.blocks():
            s += B.sum(axis=0)
        c0 = s / self.m
        r = np.zeros(self.n)
        for _, _, B in self.blocks():
            r += (B - c0[None, :]).sum(axis=0)
        self.shift = saved
        return c0 + r / self.m

    # Products by row blocks, Section 4.2.
    def times(self, X):
        """A X (m x p): each row block times X, stored in place."""
        out = np.empty((self.m, X.shape[1]))
        for r0, r1, B in self.blocks():
            out[r0:r1] = B @ X
        return out

    def t_times(self, Y):
        """A^T Y (n x p): initialise to zero, add each block's transpose
        weighted by the matching rows of Y."""
        out = np.zeros((self.n, Y.shape[1]))
        for r0, r1, B in self.blocks():
            out += B.T @ Y[r0:r1]
        return out


# ----------------------------------------------------------------------------
# Step 2: QR with column pivoting (Golub & Van Loan, Algorithm 5.4.1)
# ----------------------------------------------------------------------------
def _householder(x):
    """Householder vector v (v[0] = 1) and beta with (I - beta v v^T) x = -+||x|| e1."""
    x = np.asarray(x, dtype=np.float64)
    alpha = np.linalg.norm(x)
    v = x.copy()
    if alpha == 0.0:
        v[:] = 0.0
        v[0] = 1.0
        return v, 0.0
    s = -1.0 if x[0] < 0 else 1.0
    v[0] = x[0] + s * alpha
    v = v / v[0]
    beta = 2.0 / (v @ v)
    return v, beta


def pivoted_qr(H):
    """Householder QR with column pivoting: H P = Q R.

    Returns (Q, R, perm) with Q m x w orthonormal (all w = H.shape[1] columns
    kept, as Step 2 keeps all (i+1)l), R w x w upper triangular with
    non-increasing |R_jj|, and perm the column permutation."""
    A = np.array(H, dtype=np.float64, copy=True)
    m, w = A.shape
    if w > m:
        raise ValueError("pivoted_qr needs m >= w")
    perm = np.arange(w)
    vs, betas = [], []
    for r in range(w):
        # column norms of the trailing submatrix (recomputed, not downdated)
        c = np.einsum("ij,ij->j", A[r:, r:], A[r:, r:])
        j = r + int(np.argmax(c))
        if j != r:
            A[:, [r, j]] = A[:, [j, r]]
            perm[[r, j]] = perm[[j, r]]
        v, beta = _householder(A[r:, r])
        if beta != 0.0:
            A[r:, r:] -= beta * np.outer(v, v @ A[r:, r:])
        vs.append(v)
        betas.append(beta)
    # Q = (product of reflectors) applied to the first w columns of I
    Q = np.zeros((m, w))
    Q[:w, :w] = np.eye(w)
    for r in range(w - 1, -1, -1):
        v, beta = vs[r], betas[r]
        if beta != 0.0:
            Q[r:, :] -= beta * np.outer(v, v @ Q[r:, :])
    R = np.triu(A[:w, :w])
    return Q, R, perm


def orth(F):
    """Q factor of the thin QR of F with diag(R) >= 0 (unique for full rank)."""
    Qf, Rf = np.linalg.qr(F)
    sgn = np.where(np.diag(Rf) < 0, -1.0, 1.0)
    return Qf * sgn[None, :]


# ----------------------------------------------------------------------------
# The algorithm
# ----------------------------------------------------------------------------
def rpca(A, k, l, i, G=None, seed=None, center=False, normalize=False,
         m=None, n=None, block_rows=8192, col_scale=None, return_parts=False,
         reorth=False):
    """Rank-k approximation A ~ U diag(S) V^T by Section 3's Steps 1-6.

    A        ndarray (m x n) or callable rows(r0, r1) (then give m, n)
    G        n x l Gaussian test matrix; if None it is drawn from ``seed``
             with the Philox stream of oracle.philox (domain 0)
    center   subtract the column means first (Section 1)
    Returns U (m x k), S (k,), V (n x k) in FP64, and with return_parts a
    dict holding H blocks, Q, T and the centring vector."""
    if not callable(A):
        A = np.asarray(A)
        m, n = A.shape
    check_parameters(m, n, k, l, i)
    if n > m:
        # Section 3: apply the algorithm to A^T, then swap the factors.
        # Column operations on A (scales, centring) become row operations on
        # A^T, so they are applied here to a materialised FP64 copy.
        if callable(A):
            raise ValueError("n > m needs an ndarray A")
        At = np.asarray(A, dtype=np.float64)
        if col_scale is not None:
            At = At * np.asarray(col_scale, np.float64)[None, :]
        if center:
            At = At - At.mean(axis=0, keepdims=True)
        U, S, V, parts = _rpca_tall(At.T.copy(), k, l, i, G, seed,
                                    normalize=normalize, block_rows=block_rows,
                                    reorth=reorth)
        parts["transposed"] = True
        return (V, S, U, parts) if return_parts else (V, S, U)
    U, S, V, parts = _rpca_tall(A, k, l, i, G, seed, center=center,
                                normalize=normalize, block_rows=block_rows,
                                col_scale=col_scale, m=m, n=n, reorth=reorth)
    parts["transposed"] = False
    return (U, S, V, parts) if return_parts else (U, S, V)


def _rpca_tall(A, k, l, i, G, seed, center=False, normalize=False,
               block_rows=8192, col_scale=None, m=None, n=None, reorth=False):
    src = RowSource(A, m=m, n=n, block_rows=block_rows, col_scale=col_scale)
    if center:
        src.shift = src.column_means()
    m, n = src.m, src.n
    w = (i + 1) * l
    if G is None:
        if seed is None:
            raise ValueError("need G or seed")
        G = philox.gaussian_matrix(seed, n, l)
    G = np.asarray(G, dtype=np.float64)
    if G.shape != (n, l):
        raise ValueError("G must be n x l")

    # Step 1 (eqs. first_prod .. last_prod, product23)
    blocks = []
    X = orth(G) if reorth else G
    earlier = [X]
    for j in range(i + 1):
        Hj = src.times(X)                     # H^(j) = A X
        blocks.append(Hj)
        if j < i:
            F = src.t_times(Hj)               # F = A^T H^(j)
            if reorth:
                P = np.hstack(earlier)
                for _twice in range(2):
                    F = F - P @ (P.T @ F)     # out of span(X^(0..j))
                X = orth(F)
                earlier.append(X)
            else:
                X = orth(F) if normalize else F   # H^(j+1) = A F
    H = np.hstack(blocks)
    # Step 2 (eq. good_approx23)
    Q, R, perm = pivoted_qr(H)
    # Step 3 (eq. product_t3)
    T = src.t_times(Q)
    # Step 4 (eq. svd_small3): T = V~ Sigma~ W^T, descending
    Vt, St, WT = np.linalg.svd(T, full_matrices=False)
    W = WT.T
    # Step 5 (eq. product33)
    Ut = Q @ W
    # Step 6
    U, S, V = Ut[:, :k], St[:k], Vt[:, :k]
    parts = dict(H=blocks, Q=Q, R=R, perm=perm, T=T, W=W, S_all=St, G=G,
                 shift=src.shift)
    return U, S, V, parts


# ----------------------------------------------------------------------------
# Single products, for checking one streamed pass at a time
# ----------------------------------------------------------------------------
def fused_pass_products(A, X, shift=None, col_scale=None):
    """One streamed pass of Step 1: H = A_c X and F = A_c^T H (Section 4.2,
    'forming F = A^T H^(0) first, and H^(1) = A F second', here with the
    roles of one pass: the H it forms and the F = A^T H the next pass needs).
    A_c = A diag(col_scale) - 1 shift^T."""
    src = RowSource(A, col_scale=col_scale)
    if shift is not None:
        src.shift = np.asarray(shift, np.float64)
    H = src.times(np.asarray(X, np.float64))
    F = src.t_times(H)
    return H, F


def t_pass_product(A, Q, shift=None, col_scale=None):
    """Step 3 (eq. product_t3): T = A_c^T Q."""
    src = RowSource(A, col_scale=col_scale)
    if shift is not None:
        src.shift = np.asarray(shift, np.float64)
    return src.t_times(np.asarray(Q, np.float64))
