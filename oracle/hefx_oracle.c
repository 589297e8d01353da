/*
 * hefx oracle -- TEST INFRASTRUCTURE ONLY.
 *
 * A plain, slow, obviously-correct CPU statement of what the hefx hot path computes,
 * written from the paper (arXiv 2501.07047, "CROSS") and the textbook definitions it
 * relies on.  Only tests/, __graft_entry__.smoke() and bench.py's CPU-baseline leg may
 * load this library.  It shares no code, table or constant with the CUDA library: every
 * quantity (primitive roots, psi, inverses, basis-conversion constants) is recomputed here
 * from its definition with 64-bit values, 128-bit products and the `%` operator.  There is
 * no Montgomery, Barrett, Shoup, digit split, four-step or any other fast reduction here.
 *
 * Conventions (readings taken where the paper is silent or garbled):
 *  - ring R_q = Z_q[x]/(x^N + 1), N = 2^logn (Sec. II-A);
 *  - psi = g^((q-1)/(2N)) mod q with g the smallest generator of Z_q^* (the paper does not
 *    say how roots are chosen);
 *  - forward NTT output in bit-reversed order (Sec. IV-B2):
 *        ahat[p] = sum_j a_j * psi^(j * (2*brv_N(p) + 1))  mod q,
 *    i.e. ahat[p] = a(psi^(2 brv(p) + 1));
 *  - inverse NTT: a_j = N^-1 * sum_p ahat[p] * psi^(-j (2 brv(p) + 1)) mod q;
 *  - basis conversion exactly as written in App. B (BConv), without any correction of the
 *    multiple of Q that the fast conversion may add;
 *  - ModDown, Rescale and the key-switching inner product (the HE operators of Sec. V-A and
 *    the hybrid key switching with dnum digits of Sec. V-C, whose formulas the paper does
 *    not print) as in textbook RNS-CKKS: ModDown(x) = (x_Q - BConv_{P->Q}(x_P)) * P^-1,
 *    Rescale(x)_i = (x_i - x_{L-1}) * q_{L-1}^-1, both on coefficient-form residues.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

typedef unsigned __int128 u128;

static uint64_t mulmod(uint64_t a, uint64_t b, uint64_t q) { return (uint64_t)(((u128)a * b) % q); }

uint64_t or_powmod(uint64_t a, uint64_t e, uint64_t q) {
    uint64_t r = 1 % q;
    a %= q;
    while (e) {
        if (e & 1) r = mulmod(r, a, q);
        a = mulmod(a, a, q);
        e >>= 1;
    }
    return r;
}

/* Trial division: plain and certain for the 28-32-bit moduli used here. */
int or_is_prime(uint64_t n) {
    if (n < 2) return 0;
    if (n % 2 == 0) return n == 2;
    for (uint64_t d = 3; d * d <= n; d += 2)
        if (n % d == 0) return 0;
    return 1;
}

/* Smallest generator of the multiplicative group mod the prime q. */
uint64_t or_primitive_root(uint64_t q) {
    uint64_t f[64];
    int nf = 0;
    uint64_t m = q - 1;
    for (uint64_t d = 2; d * d <= m; ++d) {
        if (m % d == 0) {
            f[nf++] = d;
            while (m % d == 0) m /= d;
        }
    }
    if (m > 1) f[nf++] = m;
    for (uint64_t g = 2; g < q; ++g) {
        int ok = 1;
        for (int i = 0; i < nf && ok; ++i)
            if (or_powmod(g, (q - 1) / f[i], q) == 1) ok = 0;
        if (ok) return g;
    }
    return 0;
}

/* Primitive 2N-th root of unity psi; returns 0 when 2N does not divide q-1. */
uint64_t or_psi(uint64_t q, uint64_t n) {
    if ((q - 1) % (2 * n) != 0) return 0;
    return or_powmod(or_primitive_root(q), (q - 1) / (2 * n), q);
}

uint64_t or_inverse(uint64_t a, uint64_t q) { return or_powmod(a, q - 2, q); } /* q prime */

uint32_t or_bitrev(uint32_t x, int bits) {
    uint32_t r = 0;
    for (int i = 0; i < bits; ++i) r |= ((x >> i) & 1u) << (bits - 1 - i);
    return r;
}

/* ------------------------------------------------------------------ NTT, by definition */

/* One forward output: ahat[p] = sum_j a_j psi^(j(2 brv(p)+1)). O(N). */
uint32_t or_ntt_direct_at(int logn, uint64_t q, uint64_t psi, const uint32_t* a, uint32_t p) {
    uint64_t n = 1ull << logn;
    uint64_t x = or_powmod(psi, 2ull * or_bitrev(p, logn) + 1, q); /* evaluation point */
    /* Horner: a(x) = (...(a_{N-1} x + a_{N-2}) x + ...) x + a_0 */
    uint64_t acc = 0;
    for (uint64_t j = n; j-- > 0;) acc = (mulmod(acc, x, q) + a[j]) % q;
    return (uint32_t)acc;
}

/* One inverse output: a_j = N^-1 sum_p ahat[p] psi^(-j(2 brv(p)+1)). O(N log q). */
uint32_t or_intt_direct_at(int logn, uint64_t q, uint64_t psi, const uint32_t* ahat, uint32_t j) {
    uint64_t n = 1ull << logn;
    uint64_t psi_inv = or_inverse(psi, q);
    u128 acc = 0;
    for (uint64_t p = 0; p < n; ++p) {
        uint64_t e = ((uint64_t)j * (2ull * or_bitrev((uint32_t)p, logn) + 1)) % (2 * n);
        acc += (u128)ahat[p] * or_powmod(psi_inv, e, q);
        acc %= q;
    }
    return (uint32_t)mulmod((uint64_t)acc, or_inverse(n % q, q), q);
}

/* Full O(N^2) forward transform by the definition. */
void or_ntt_direct(int logn, uint64_t q, uint64_t psi, const uint32_t* a, uint32_t* out) {
    uint64_t n = 1ull << logn;
    for (uint64_t p = 0; p < n; ++p) out[p] = or_ntt_direct_at(logn, q, psi, a, (uint32_t)p);
}

/* ------------------------------------------------------------------ NTT, O(N log N)
 * The same definition evaluated fast: with omega = psi^2,
 *     ahat[brv(k)] = sum_j (a_j psi^j) omega^(j k),
 * i.e. a pre-twist by psi^j followed by a cyclic length-N DFT over Z_q (computed by the
 * iterative radix-2 algorithm on bit-reversed input) whose k-th output is stored at
 * position brv(k).  The inverse undoes each of these steps in reverse order. */

static void cyclic_dft(int logn, uint64_t q, uint64_t omega, uint64_t* x) {
    uint64_t n = 1ull << logn;
    for (uint64_t i = 0; i < n; ++i) { /* bit-reversal permutation of the input */
        uint64_t r = or_bitrev((uint32_t)i, logn);
        if (r > i) { uint64_t t = x[i]; x[i] = x[r]; x[r] = t; }
    }
    for (uint64_t len = 2; len <= n; len <<= 1) {
        uint64_t w_len = or_powmod(omega, n / len, q);
        for (uint64_t s = 0; s < n; s += len) {
            uint64_t w = 1;
            for (uint64_t i = 0; i < len / 2; ++i) {
                uint64_t u = x[s + i], v = mulmod(x[s + i + len / 2], w, q);
                x[s + i] = (u + v) % q;
                x[s + i + len / 2] = (u + q - v) % q;
                w = mulmod(w, w_len, q);
            }
        }
    }
}

void or_ntt_fwd(int logn, uint64_t q, uint64_t psi, uint32_t* a) {
    uint64_t n = 1ull << logn;
    uint64_t* x = (uint64_t*)malloc(n * sizeof(uint64_t));
    uint64_t pw = 1;
    for (uint64_t j = 0; j < n; ++j) { x[j] = mulmod(a[j], pw, q); pw = mulmod(pw, psi, q); }
    cyclic_dft(logn, q, mulmod(psi, psi, q), x);
    for (uint64_t k = 0; k < n; ++k) a[or_bitrev((uint32_t)k, logn)] = (uint32_t)x[k];
    free(x);
}

void or_ntt_inv(int logn, uint64_t q, uint64_t psi, uint32_t* a) {
    uint64_t n = 1ull << logn;
    uint64_t* x = (uint64_t*)malloc(n * sizeof(uint64_t));
    uint64_t psi_inv = or_inverse(psi, q);
    for (uint64_t k = 0; k < n; ++k) x[k] = a[or_bitrev((uint32_t)k, logn)];
    cyclic_dft(logn, q, mulmod(psi_inv, psi_inv, q), x);
    uint64_t n_inv = or_inverse(n % q, q), pw = n_inv;
    for (uint64_t j = 0; j < n; ++j) { a[j] = (uint32_t)mulmod(x[j], pw, q); pw = mulmod(pw, psi_inv, q); }
    free(x);
}

/* Rows of a [rows][N] array, row r modulo qs[r] (psi recomputed per distinct modulus). */
void or_ntt_rows(int logn, int inverse, size_t rows, const uint32_t* qs, uint32_t* data) {
    uint64_t n = 1ull << logn, last_q = 0, psi = 0;
    for (size_t r = 0; r < rows; ++r) {
        if (qs[r] != last_q) { last_q = qs[r]; psi = or_psi(last_q, n); }
        if (inverse) or_ntt_inv(logn, last_q, psi, data + r * n);
        else or_ntt_fwd(logn, last_q, psi, data + r * n);
    }
}

/* ------------------------------------------------------------------ polynomial product */

/* Schoolbook negacyclic product c = a*b mod (x^N + 1, q): x^N = -1 wraps with a minus. */
void or_polymul_schoolbook(int logn, uint64_t q, const uint32_t* a, const uint32_t* b, uint32_t* c) {
    uint64_t n = 1ull << logn;
    for (uint64_t k = 0; k < n; ++k) {
        u128 pos = 0, neg = 0;
        for (uint64_t i = 0; i <= k; ++i) pos += (u128)a[i] * b[k - i];
        for (uint64_t i = k + 1; i < n; ++i) neg += (u128)a[i] * b[n + k - i];
        uint64_t p = (uint64_t)(pos % q), m = (uint64_t)(neg % q);
        c[k] = (uint32_t)((p + q - m) % q);
    }
}

/* The product the hot path computes: INTT(NTT(a) o NTT(b)). */
void or_polymul_ntt(int logn, uint64_t q, uint64_t psi, const uint32_t* a, const uint32_t* b, uint32_t* c) {
    uint64_t n = 1ull << logn;
    uint32_t* t = (uint32_t*)malloc(n * sizeof(uint32_t));
    memcpy(c, a, n * sizeof(uint32_t));
    memcpy(t, b, n * sizeof(uint32_t));
    or_ntt_fwd(logn, q, psi, c);
    or_ntt_fwd(logn, q, psi, t);
    for (uint64_t i = 0; i < n; ++i) c[i] = (uint32_t)mulmod(c[i], t[i], q);
    or_ntt_inv(logn, q, psi, c);
    free(t);
}

void or_polymul_rows(int logn, size_t rows, const uint32_t* qs, const uint32_t* a, const uint32_t* b, uint32_t* c) {
    uint64_t n = 1ull << logn, last_q = 0, psi = 0;
    for (size_t r = 0; r < rows; ++r) {
        if (qs[r] != last_q) { last_q = qs[r]; psi = or_psi(last_q, n); }
        or_polymul_ntt(logn, last_q, psi, a + r * n, b + r * n, c + r * n);
    }
}

/* ------------------------------------------------------------------ basis conversion
 * App. B:  Conv(a)_{n,j} = sum_i [a_{n,i} * qhat_i^-1]_{q_i} * [qhat_i]_{p_j}  mod p_j,
 * qhat_i = Q / q_i = prod_{k != i} q_k.  in: [L][n], out: [Lp][n]. */
void or_bconv(size_t n, int L, const uint32_t* qs, int Lp, const uint32_t* ps, const uint32_t* in, uint32_t* out) {
    uint64_t* qhat_inv = (uint64_t*)malloc(sizeof(uint64_t) * L);
    uint64_t* qhat_p = (uint64_t*)malloc(sizeof(uint64_t) * L * Lp);
    for (int i = 0; i < L; ++i) {
        uint64_t h = 1;
        for (int k = 0; k < L; ++k) if (k != i) h = mulmod(h, qs[k], qs[i]);
        qhat_inv[i] = or_inverse(h, qs[i]);
        for (int j = 0; j < Lp; ++j) {
            uint64_t hp = 1;
            for (int k = 0; k < L; ++k) if (k != i) hp = mulmod(hp, qs[k], ps[j]);
            qhat_p[i * Lp + j] = hp;
        }
    }
    for (size_t x = 0; x < n; ++x) {
        for (int j = 0; j < Lp; ++j) {
            u128 acc = 0;
            for (int i = 0; i < L; ++i) {
                uint64_t b = mulmod(in[(size_t)i * n + x], qhat_inv[i], qs[i]); /* step 1 */
                acc += (u128)b * qhat_p[i * Lp + j];                          /* step 2 */
            }
            out[(size_t)j * n + x] = (uint32_t)(acc % ps[j]);
        }
    }
    free(qhat_inv);
    free(qhat_p);
}

/* ------------------------------------------------------------------ modular matmul
 * Z = A @ B mod q for A: H x V, B: V x W (row-major), the operation of Alg. 2. */
void or_modmatmul(size_t H, size_t V, size_t W, uint64_t q, const uint32_t* A, const uint32_t* B, uint32_t* Z) {
    for (size_t h = 0; h < H; ++h)
        for (size_t w = 0; w < W; ++w) {
            u128 acc = 0;
            for (size_t v = 0; v < V; ++v) acc += (u128)A[h * V + v] * B[v * W + w];
            Z[h * W + w] = (uint32_t)(acc % q);
        }
}

/* ------------------------------------------------------------------ key switching pieces
 * ModDown: x is [L + K][n] (Q limbs q_0..q_{L-1}, then P limbs p_0..p_{K-1}), coefficient
 * form.  out_j = (x_j - BConv_{P->Q}(x_P)_j) * P^-1 mod q_j, P = prod p_k.  out: [L][n]. */
void or_moddown(size_t n, int L, const uint32_t* qs, int K, const uint32_t* ps, const uint32_t* x, uint32_t* out) {
    uint32_t* y = (uint32_t*)malloc(sizeof(uint32_t) * (size_t)L * n);
    or_bconv(n, K, ps, L, qs, x + (size_t)L * n, y);
    for (int j = 0; j < L; ++j) {
        uint64_t P = 1;
        for (int k = 0; k < K; ++k) P = mulmod(P, ps[k], qs[j]);
        const uint64_t pinv = or_inverse(P, qs[j]);
        for (size_t c = 0; c < n; ++c) {
            const uint64_t d = (x[(size_t)j * n + c] + (uint64_t)qs[j] - y[(size_t)j * n + c] % qs[j]) % qs[j];
            out[(size_t)j * n + c] = (uint32_t)mulmod(d, pinv, qs[j]);
        }
    }
    free(y);
}

/* Rescale: x is [L][n] coefficient form over q_0..q_{L-1}.
 * out_i = (x_i - (x_{L-1} mod q_i)) * q_{L-1}^-1 mod q_i for i < L - 1.  out: [L-1][n]. */
void or_rescale(size_t n, int L, const uint32_t* qs, const uint32_t* x, uint32_t* out) {
    const uint64_t ql = qs[L - 1];
    for (int i = 0; i < L - 1; ++i) {
        const uint64_t inv = or_inverse(ql % qs[i], qs[i]);
        for (size_t c = 0; c < n; ++c) {
            const uint64_t last = x[(size_t)(L - 1) * n + c] % qs[i];
            const uint64_t d = (x[(size_t)i * n + c] + (uint64_t)qs[i] - last) % qs[i];
            out[(size_t)i * n + c] = (uint32_t)mulmod(d, inv, qs[i]);
        }
    }
}

/* Key-switching inner product: digits [dnum][nl][n], evk [dnum][2][nl][n] (limb l reduced
 * by qs[l]); out[k][l][c] = sum_j digits[j][l][c] * evk[j][k][l][c] mod qs[l], k = 0, 1. */
void or_key_inner_product(size_t n, int nl, const uint32_t* qs, int dnum, const uint32_t* digits, const uint32_t* evk,
                          uint32_t* out) {
    for (int k = 0; k < 2; ++k)
        for (int l = 0; l < nl; ++l)
            for (size_t c = 0; c < n; ++c) {
                u128 acc = 0;
                for (int j = 0; j < dnum; ++j)
                    acc += (u128)digits[((size_t)j * nl + l) * n + c] * evk[(((size_t)j * 2 + k) * nl + l) * n + c];
                out[((size_t)k * nl + l) * n + c] = (uint32_t)(acc % qs[l]);
            }
}
