"""The BAT constructions of the paper, in plain Python integers -- TEST INFRASTRUCTURE ONLY.

These are not used to check GPU outputs (the GPU's modular products are checked against
the plain definitions in `hefx_oracle.c`).  They pin this project's reading of BAT
(Sec. IV-A2 and Alg. 2): a known factor `a` times a runtime value `b` split into
chunks b_j of `w` bits equals, modulo q,

    sum_i 2^(w' i) * sum_j M[i][j] * b_j ,   M[i][j] = chunk'_i((a * 2^(w j)) mod q),

where chunk'_i takes `w'`-bit chunks.  Alg. 2 uses w = w' = bp; the derivation of
Sec. IV-A2 holds for any pair of widths.  Eqs. (1)-(5) print the shift of chunk i as
2^i; the derivation needs 2^(bp i), which is the reading taken here.
"""
from __future__ import annotations


def chunk_decompose(a: int, bits: int, count: int) -> list[int]:
    """ChunkDecompose of Alg. 2: chunk k = (a >> k*bits) & (2^bits - 1)."""
    mask = (1 << bits) - 1
    return [(int(a) >> (k * bits)) & mask for k in range(count)]


def chunk_merge(chunks, bits: int) -> int:
    """ChunkMerge of Alg. 2: sum_k chunk_k << k*bits (plain integers, no reduction)."""
    return sum(int(c) << (k * bits) for k, c in enumerate(chunks))


def direct_scalar_bat(a: int, q: int, w: int, k_in: int, w_out: int | None = None,
                      k_out: int | None = None) -> list[list[int]]:
    """DirectScalarBAT of Alg. 2: column j holds the w_out-bit chunks of (a << j*w) mod q."""
    w_out = w if w_out is None else w_out
    k_out = k_in if k_out is None else k_out
    M = [[0] * k_in for _ in range(k_out)]
    for j in range(k_in):
        val = (int(a) << (j * w)) % q
        for i, c in enumerate(chunk_decompose(val, w_out, k_out)):
            M[i][j] = c
        assert chunk_merge(chunk_decompose(val, w_out, k_out), w_out) == val
    return M


def offline_compile_left(A, q: int, w: int, k_in: int, w_out=None, k_out=None):
    """OfflineCompileLeft of Alg. 2: embed the k_out x k_in block of each A[h][v]."""
    k_out = k_in if k_out is None else k_out
    H, V = len(A), len(A[0])
    D = [[0] * (V * k_in) for _ in range(H * k_out)]
    for h in range(H):
        for v in range(V):
            M = direct_scalar_bat(A[h][v], q, w, k_in, w_out, k_out)
            for i in range(k_out):
                for j in range(k_in):
                    D[h * k_out + i][v * k_in + j] = M[i][j]
    return D


def runtime_compile_right(B, w: int, k_in: int):
    """RuntimeCompileRight of Alg. 2: stack the w-bit chunks of B[v][w] vertically."""
    V, W = len(B), len(B[0])
    D = [[0] * W for _ in range(V * k_in)]
    for v in range(V):
        for col in range(W):
            for k, c in enumerate(chunk_decompose(B[v][col], w, k_in)):
                D[v * k_in + k][col] = c
    return D


def bat_modmatmul(A, B, q: int, w: int, k_in: int, w_out=None, k_out=None):
    """Main-FullMatMul of Alg. 2 followed by the final reduction mod q.

    Returns (Z mod q, max partial sum) -- the second value is the largest entry of the
    low-precision product, i.e. the accumulator range the matrix engine must hold."""
    w_out = w if w_out is None else w_out
    k_out = k_in if k_out is None else k_out
    Ad = offline_compile_left(A, q, w, k_in, w_out, k_out)
    Bd = runtime_compile_right(B, w, k_in)
    H, W = len(A), len(B[0])
    KV = len(Bd)
    Zc = [[sum(Ad[r][k] * Bd[k][c] for k in range(KV)) for c in range(W)] for r in range(H * k_out)]
    peak = max(max(row) for row in Zc)
    Z = [[chunk_merge([Zc[h * k_out + i][c] for i in range(k_out)], w_out) % q for c in range(W)]
         for h in range(H)]
    return Z, peak


# ----------------------------------------------------------------------------- Alg. 5

def iterative_scalar_bat(a: int, q: int, bp: int, K: int, max_rounds: int = 64):
    """The offline construction of Alg. 5: start from the (2K-1) x K Toeplitz matrix of the
    chunks of `a` (entry [i+j][j] = a_i, weight 2^(bp*row)), fold every entry of a row
    >= K back into rows < K of the same column as the chunks of (entry << bp*row) mod q,
    and propagate carries so every entry is below 2^bp, until the bottom block is zero.

    The printed pseudocode indexes the fold target column as K-1-j and limits the chunk
    loop to k < 3; both are read here as "same column" and "k < K" (the column-sum
    invariant below only holds that way)."""
    a_chunks = chunk_decompose(a, bp, K)
    rows = 2 * K - 1
    X = [[0] * K for _ in range(rows)]
    for j in range(K):
        for i in range(K):
            X[i + j][j] = a_chunks[i]
    mask = (1 << bp) - 1
    for _ in range(max_rounds):
        # carry propagation (may spill into rows >= K, which are folded below)
        for j in range(K):
            for r in range(rows):
                if X[r][j] > mask:
                    c = X[r][j] >> bp
                    X[r][j] &= mask
                    if r + 1 == rows:
                        X.append([0] * K)
                        rows += 1
                    X[r + 1][j] += c
        if all(X[r][j] == 0 for r in range(K, rows) for j in range(K)):
            return [row[:] for row in X[:K]]
        # fold the bottom block
        for j in range(K):
            for r in range(K, rows):
                if X[r][j]:
                    proj = (X[r][j] << (bp * r)) % q
                    X[r][j] = 0
                    for k, c in enumerate(chunk_decompose(proj, bp, K)):
                        X[k][j] += c
    raise RuntimeError("iterative BAT did not converge")
