/*
 * hefx -- batched negacyclic NTT, polynomial product and RNS basis conversion on one
 * NVIDIA GB300 (sm_103a), after arXiv 2501.07047 ("CROSS").
 *
 * Conventions shared by every call
 * --------------------------------
 *  - A polynomial in R_Q = Z_Q[x]/(x^N + 1) (Sec. II-A) is held in RNS form (Sec. II-A,
 *    "Residue Number System"): one limb of N residues per prime q_i.  Device buffers are
 *    uint32 arrays laid out [batch][limb][N], row-major, contiguous, 16-byte aligned, every
 *    value a canonical residue in [0, q_limb).  Inputs outside [0, q) give undefined
 *    (but memory-safe) results.
 *  - The forward NTT maps coefficient order to evaluation order with the output in
 *    bit-reversed order (Sec. IV-B2, "layout invariant 3-step negacyclic NTT"):
 *        ahat[p] = sum_j a_j * psi^(j (2 brv_N(p) + 1))  mod q,
 *    psi = g^((q-1)/(2N)), g the smallest generator of Z_q^*.  The inverse NTT maps
 *    bit-reversed evaluations back to natural-order coefficients and includes N^-1.
 *  - Every call is asynchronous on `stream` (a cudaStream_t passed as void*, NULL = the
 *    legacy default stream).  Errors that the host can detect are returned synchronously
 *    and nothing is launched; hefx_last_error() then holds a one-line message.  Most
 *    kernels launch with programmatic stream serialization: their set-up may overlap the
 *    drain of the stream's preceding kernel, and each waits for that kernel to complete
 *    before touching memory, so the ordering against earlier stream work is unchanged.
 *  - Tensor-path transforms keep a digit workspace in their parameter set: tensor-path calls
 *    with the same params whose work overlaps on the GPU (different streams) race on it.
 *    Issue them on one stream, or give each stream its own parameter set.  The CUDA-core
 *    kernels keep no state between launches, and their calls may overlap freely.
 *  - The caller owns every data buffer (device pointers from any allocator).  hefx owns
 *    the context, parameter sets and plans it creates (and the device tables inside them),
 *    and releases them in the matching *_destroy call.
 *  - Moduli: primes q with q = 1 (mod 2N) and 2^3 < q < 2^30 (the lazy butterflies keep
 *    values below 4q < 2^32).  N = 2^log2n with 3 <= log2n <= 17 (the tensor path covers
 *    12 <= log2n <= 16, with moduli above 2^28 all of them but 2^13; N = 2^17 needs
 *    q = 1 mod 2^18 and runs on the CUDA cores).
 *  - Paths: HEFX_PATH_CUDACORE is the radix-2 Cooley-Tukey / Gentleman-Sande transform on
 *    the CUDA cores (App. A, "Radix-2 Cooley-Tukey NTT").  HEFX_PATH_TENSOR is the
 *    layout-invariant matrix NTT of Sec. IV-B with its modular matrix products split into
 *    small-integer digits (BAT, Sec. IV-A) and run on the tcgen05 tensor cores.
 *    HEFX_PATH_AUTO takes the path the built-in tuner measured fastest for the shape.
 *    Both paths return identical (bit-exact) results.
 */
#ifndef HEFX_H
#define HEFX_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    HEFX_OK = 0,
    HEFX_EINVAL = 1,       /* a bad argument: null pointer, bad prime, misaligned buffer */
    HEFX_EUNSUPPORTED = 2, /* a valid request outside what this build implements */
    HEFX_ENOMEM = 3,       /* a device allocation for tables or workspace failed */
    HEFX_EBUDGET = 4,      /* a request does not fit the configured memory budget */
    HEFX_ECUDA = 5,        /* a CUDA runtime call failed (message in hefx_last_error) */
    HEFX_ETIMEOUT = 6      /* a bounded device-side wait expired; results are invalid */
} hefx_status;

typedef enum {
    HEFX_PATH_AUTO = 0,
    HEFX_PATH_CUDACORE = 1,
    HEFX_PATH_TENSOR = 2
} hefx_path;

typedef struct hefx_ctx hefx_ctx;
typedef struct hefx_params hefx_params;
typedef struct hefx_bconv_plan hefx_bconv_plan;
typedef struct hefx_modup_plan hefx_modup_plan;

/* Creates a context bound to CUDA device `device` (made current by every hefx call). */
hefx_status hefx_create(hefx_ctx** out, int device);
void hefx_destroy(hefx_ctx* ctx);
/* Message of the last failed call on this context ("" when none); owned by the context. */
const char* hefx_last_error(const hefx_ctx* ctx);
/* Library version string, static storage. */
const char* hefx_version(void);

/*
 * Parameter set for N = 2^log2n and the RNS basis primes[0..nlimbs) (Sec. II-A; Table
 * "Notations": q_i coprime, L limbs).  Precomputes on the host and uploads the twiddle
 * tables of both paths (the offline "compile time" step of Sec. IV-A/IV-B).
 * Errors: EINVAL for a non-prime, repeated prime, q != 1 mod 2N or q >= 2^30;
 * EUNSUPPORTED for log2n outside [3, 17]; ENOMEM when the tables do not fit.
 */
hefx_status hefx_params_create(hefx_ctx* ctx, uint32_t log2n, const uint32_t* primes, uint32_t nlimbs,
                               hefx_params** out);
void hefx_params_destroy(hefx_params* params);

/*
 * Records the path HEFX_PATH_AUTO takes for this parameter set (HEFX_PATH_CUDACORE or
 * HEFX_PATH_TENSOR; HEFX_PATH_AUTO restores the default, the CUDA-core path).  Called by
 * the autotuner after it has timed both paths on the device (Sec. V-B3 reports the best
 * of several (R, C) splits per shape; the tuner generalises that choice).
 * Errors: EINVAL for a null params or an unknown path.  Not thread-safe with concurrent
 * calls that use the same params.
 */
hefx_status hefx_params_set_auto_path(hefx_params* params, hefx_path path);

/*
 * Tensor-path configuration of a parameter set, for the autotuner (Sec. V-A sweeps the
 * (R, C) split of each operator; deeper splits and the GEMM tile are this library's own):
 *  - log2r2 == 0: the matrix NTT's split N = R x C with R = 2^log2r (0: R = 2^floor(log2n /
 *    2)); both R and C must be 64 .. 256: the transposing digit split works on 64-wide tiles,
 *    and the fp32 accumulation of 7-bit digit products stays exact only for reduction lengths
 *    up to 256 (a step with 64 data rows per limb packs two polynomials into one of the GEMM's
 *    128-row blocks).  So N = 2^12 has one such split, 2^13 two, 2^14 three, 2^15 two, 2^16
 *    one.
 *  - log2r2 > 0: three factors N = R1 x R2 x R3, R1 = 2^log2r (64 .. 256: the transposing
 *    digit split works on 64-wide tiles), R2 = 2^log2r2 and R3 = N / (R1 R2) (16 .. 256): step
 *    1 over R1 as before, then the remaining cyclic transform of each row as two digit GEMMs
 *    (R2, then R3) with a twiddle between them.  Fewer digit MACs (16 N (R1 + R2 + R3) instead of
 *    16 N (R + C)), one more epilogue.
 *  - tile_outputs: outputs per GEMM tile, 64 (256 accumulator columns) or 32 (128); steps with
 *    fewer outputs take a tile of their output count (16 or 32).
 *  - A parameter set with a modulus of 29 or 30 bits runs the tensor path on 8-bit digits and
 *    chunks, whose fp32 sums stay exact only for reduction lengths up to 64 (4 * 64 * 255 *
 *    255 < 2^24): it takes splits with every factor at most 64 (R1 = 64; its default is 64 x 64
 *    at N = 2^12, 64 x 32 x 32 at 2^16, 64 x 32 x 16 at 2^15, 64 x 16 x 16 at 2^14; 2^13 has
 *    none and stays on the CUDA cores); other splits give EUNSUPPORTED.
 * Results do not depend on any of these choices.  Changing the split drops the parameter set's
 * pipelined tensor tables (after a device synchronization); the next tensor-path call builds
 * them for the new split.  Errors: EINVAL (no such split or tile), EUNSUPPORTED (see above),
 * ECUDA.
 */
hefx_status hefx_params_set_tensor_config(hefx_params* params, uint32_t log2r, uint32_t log2r2,
                                          uint32_t tile_outputs);

/*
 * Modular reductions of the paper's ablation (Sec. V-F, "Impact of Modular Reduction
 * Algorithm": Barrett, Montgomery, Shoup).
 */
typedef enum {
    HEFX_RED_SHOUP = 0,
    HEFX_RED_MONTGOMERY = 1,
    HEFX_RED_BARRETT = 2,
    HEFX_RED_BAT_LAZY = 3 /* VecModMul only: BAT lazy reduction on the tensor cores */
} hefx_reduction;

/*
 * Selects the reduction of the CUDA-core NTT's twiddle products (ntt_red; default Shoup) and
 * of hefx_vec_mod_mul (vec_red; default Montgomery) for this parameter set.  Montgomery
 * twiddles keep w 2^32 mod q (a second table, built here on first use); Barrett takes the
 * quotient of the 64-bit product from floor(2^64 / q).  Every choice returns the same
 * (canonical) results.  Non-default ntt_red covers hefx_ntt_fwd / hefx_ntt_inv at
 * N = 2^16 only: other sizes, hefx_poly_mul and the tensor path then return EUNSUPPORTED;
 * batch plans always use Shoup.  vec_red = HEFX_RED_SHOUP is EINVAL (Shoup needs a
 * precomputed companion of one operand; VecModMul's operands are both runtime values).
 * vec_red = HEFX_RED_BAT_LAZY (the paper's appendix "BAT for Modular Reduction", part of the
 * Sec. V-F ablation) reduces the 64-bit product's high four bytes with a byte-matrix product
 * on the tensor cores (one tcgen05 MMA per 128 elements) and finishes with one Barrett
 * reduction; it needs log2n >= 9 (EUNSUPPORTED otherwise) and is used by hefx_vec_mod_mul.
 * Synchronous; not thread-safe with concurrent calls that use the same params.
 */
hefx_status hefx_params_set_reduction(hefx_params* params, hefx_reduction ntt_red, hefx_reduction vec_red);

/*
 * Schedules of the CUDA-core NTT / INTT of contiguous rows (hefx_ntt_fwd, hefx_ntt_inv and the
 * plain transforms inside other calls).  Both run the same radix-2 butterflies (App. A) and
 * return identical results.
 *  - HEFX_CC_CLUSTER: one launch; a row of N = 2^16 is split over a cluster of 8 CTAs and
 *    its three cross-CTA stages go through distributed shared memory.
 *  - HEFX_CC_TWO_PASS (N = 2^16 only): two launches through L2, the row / column
 *    factorisation of the matrix NTT (Sec. IV-B) with the twiddle step folded into the
 *    butterflies: 8 stages within columns j mod 256, then 8 within 256-element blocks
 *    (reversed for the inverse); the intermediate goes through the output buffer.
 *  - HEFX_CC_AUTO (default): at N = 2^16, HEFX_CC_TWO_PASS for at most 32 rows (so few
 *    clusters leave most of the GPU idle; measured 20 % faster for one polynomial of 24
 *    limbs) and for one to one and a half waves of co-resident clusters (the cluster
 *    kernel's second wave mostly empty; 4-14 % faster at 96 and 120 rows), else
 *    HEFX_CC_CLUSTER.
 * Hadamard-fused forms (hefx_poly_mul), Rescale, row lists and batch plans use the cluster
 * schedule.  Errors: EINVAL (unknown schedule), EUNSUPPORTED (HEFX_CC_TWO_PASS at
 * N != 2^16).  Not thread-safe with concurrent calls that use the same params.
 */
typedef enum { HEFX_CC_AUTO = 0, HEFX_CC_CLUSTER = 1, HEFX_CC_TWO_PASS = 2 } hefx_cc_schedule;
hefx_status hefx_params_set_cc_schedule(hefx_params* params, hefx_cc_schedule schedule);

/*
 * In-place forward NTT of d_data[batch][nlimbs][N] (natural order in, bit-reversed out).
 * The definition is Sec. II-A's ring with the bit-reversed output of Sec. IV-B2; the
 * CUDA-core path follows App. A (radix-2 Cooley-Tukey), the tensor path Sec. IV-B
 * (layout-invariant 3-step NTT with BAT-split matrix products).
 * batch == 0 is a no-op.  Errors: EINVAL (null/misaligned pointer), EUNSUPPORTED (path
 * not available for this N), ECUDA (launch failure).
 */
hefx_status hefx_ntt_fwd(hefx_ctx* ctx, const hefx_params* params, uint32_t* d_data, size_t batch,
                         hefx_path path, void* stream);

/* In-place inverse NTT (bit-reversed in, natural out, scaled by N^-1); same contract. */
hefx_status hefx_ntt_inv(hefx_ctx* ctx, const hefx_params* params, uint32_t* d_data, size_t batch,
                         hefx_path path, void* stream);

/*
 * Negacyclic product c = a * b in R_q per limb (Sec. III, Table "HE operator -> AI
 * operator": NTT, Hadamard product mod q, INTT).  Inputs and output in natural
 * coefficient order, [batch][nlimbs][N].  d_c may alias d_a and/or d_b.  Uses no
 * workspace beyond d_c.  Errors as for hefx_ntt_fwd.
 */
hefx_status hefx_poly_mul(hefx_ctx* ctx, const hefx_params* params, const uint32_t* d_a, const uint32_t* d_b,
                          uint32_t* d_c, size_t batch, hefx_path path, void* stream);

/*
 * Same product as hefx_poly_mul on the tensor path, for callers that must not allocate
 * device memory once they are running: code whose memory is planned up front (a fixed arena
 * handed out by a host framework), or a latency-critical loop where a cudaMalloc could
 * block on device-wide synchronization or fail under memory pressure.  hefx_poly_mul's
 * tensor path keeps its digit workspace in the parameter set and allocates it lazily: on
 * its first call, and again (after a device synchronization) whenever a larger batch
 * arrives.  This variant never allocates, not even lazily: its workspace is a fixed 8 MiB
 * array compiled into the library (2^21 residues), which every GPU that loads the library
 * keeps until the process exits.
 * There is no counterpart in the paper: this is a deployment variant of the same math.
 *  - Calls no cudaMalloc, cudaFree or allocating library routine.  The parameter set's
 *    tensor tables must exist already: make one tensor-path call with `params` first
 *    (e.g. hefx_poly_mul with HEFX_PATH_TENSOR), else HEFX_EUNSUPPORTED.
 *  - batch * nlimbs * N must not exceed 2^21, else HEFX_EINVAL (split the batch).
 *  - The first call on each device looks up the array's device address (with that device
 *    current); make that first call before any stream capture.
 *  - All calls share the one array and it keeps the last call's contents (each call writes
 *    it fully before reading it, so nothing needs clearing).  Calls whose work overlaps on
 *    the GPU (different streams, or different host threads) race on it: serialize them.
 *  - Like hefx_poly_mul, it takes the default (Shoup) NTT reduction only: a parameter set
 *    switched to another reduction gets HEFX_EUNSUPPORTED.  It runs the single-pass tensor
 *    form, built for moduli below 2^28: a parameter set with a larger modulus gets
 *    HEFX_EUNSUPPORTED.
 *  - Layout, aliasing (d_c may alias d_a and/or d_b) and errors otherwise as for
 *    hefx_poly_mul.
 */
hefx_status hefx_poly_mul_noalloc(hefx_ctx* ctx, const hefx_params* params, const uint32_t* d_a,
                                  const uint32_t* d_b, uint32_t* d_c, size_t batch, void* stream);

/*
 * Basis-conversion plan from basis src[0..L) to basis dst[0..Lp) for limbs of
 * n = 2^log2n coefficients (App. B, BConv):
 *   out_{n,j} = sum_i [a_{n,i} * qhat_i^-1]_{q_i} * [qhat_i]_{p_j}  mod p_j,  qhat_i = Q / q_i.
 * This is the fast conversion as written: the integer it reduces may exceed the CRT value
 * by u*Q with 0 <= u < L; no correction is applied.  The plan holds the step-1 constants
 * qhat_i^-1 mod q_i and the BAT-compiled digit matrix of step 2 (Sec. IV-A3).
 * Errors: EINVAL for non-prime, repeated (within or across bases) or >= 2^30 moduli,
 * L or Lp outside [1, 64]; EUNSUPPORTED for log2n outside [0, 24] or when
 * L * max(q) * max(p) >= 2^64 (the CUDA-core kernel sums L products in 64 bits).
 */
hefx_status hefx_bconv_plan_create(hefx_ctx* ctx, uint32_t log2n, const uint32_t* src, uint32_t L,
                                   const uint32_t* dst, uint32_t Lp, hefx_bconv_plan** out);
void hefx_bconv_plan_destroy(hefx_bconv_plan* plan);

/*
 * d_out[batch][Lp][n] = BConv(d_in[batch][L][n]).  d_out must not overlap d_in.
 * HEFX_PATH_TENSOR runs step 2 as a digit-split matrix product on the tensor cores
 * (Sec. IV-A3, "High-Precision MatModMul in BConv"); HEFX_PATH_CUDACORE as 64-bit
 * multiply-accumulates (with L <= 48 and N >= 2^8, over tiles that TMA streams into shared
 * memory; both pipelined kernels report an expired bounded wait through hefx_bconv_check).
 * Results are identical.  The plan has the tensor path when every
 * source prime is below 2^28, L <= 48, Lp <= 64 (one 256-column MMA: four 8-bit chunk
 * columns per target) and the kernel's tiles fit one CTA's shared memory; otherwise
 * HEFX_PATH_TENSOR returns HEFX_EUNSUPPORTED.  HEFX_PATH_AUTO takes the tensor path only when
 * the plan has it, Lp >= 48 and batch * L * n >= 96 * 2^16 (where it measured faster: the
 * CUDA-core kernel makes one pass over the sources per 8 targets, so many targets favour the
 * matrix form); otherwise the CUDA-core path.
 */
hefx_status hefx_basis_convert(hefx_ctx* ctx, const hefx_bconv_plan* plan, const uint32_t* d_in, uint32_t* d_out,
                               size_t batch, hefx_path path, void* stream);

/*
 * Waits for `stream`, then reports whether a bounded device-side wait of the pipelined
 * conversion kernels launched with `plan` (the tensor path, and the CUDA-core path where its
 * tiles arrive by TMA: L <= 48 and N >= 2^8) expired since the last check (HEFX_ETIMEOUT; the
 * results of those calls are invalid) and clears that record, as hefx_stream_check does for
 * a parameter set.  Errors: EINVAL, ECUDA, ETIMEOUT.
 */
hefx_status hefx_bconv_check(hefx_ctx* ctx, const hefx_bconv_plan* plan, void* stream);

/*
 * ModUp of hybrid key switching (the HE-Mult / Relin. of Sec. V-A and V-C, "Effects of
 * Security Parameters", built from BConv per App. A; the formulas are textbook RNS-CKKS):
 * the ciphertext basis Q = q[0..L) is cut into dnum = ceil(L / alpha) digits D_j = limbs
 * [j alpha, min(L, (j + 1) alpha)), and digit j's polynomial is extended to Q u P (P =
 * p[0..K), appended after Q):
 *   U[b][j][l] = c[b][l]                       for l in D_j,
 *   U[b][j][l] = BConv_{D_j -> {l}}(c[b][D_j])  otherwise (the fast conversion of
 *                hefx_basis_convert, sources D_j, target limb l of Q u P).
 * hefx_modup_plan_create takes the primes (distinct primes in [3, 2^30), L + K <= 64,
 * alpha in [1, L]) and uploads every digit's constants; EUNSUPPORTED for log2n > 24 or when
 * alpha * max(q) * max(q, p) >= 2^64.  hefx_mod_up converts all digits in one launch on the
 * CUDA cores.  Layouts: d_c [batch][L][N] and d_U [batch][dnum][L + K][N], coefficient form,
 * canonical, 16-byte aligned; d_U must not overlap d_c (EINVAL).
 */
hefx_status hefx_modup_plan_create(hefx_ctx* ctx, uint32_t log2n, const uint32_t* q, uint32_t L, const uint32_t* p,
                                   uint32_t K, uint32_t alpha, hefx_modup_plan** out);
void hefx_modup_plan_destroy(hefx_modup_plan* plan);
uint32_t hefx_modup_plan_dnum(const hefx_modup_plan* plan); /* 0 for a null plan */
hefx_status hefx_mod_up(hefx_ctx* ctx, const hefx_modup_plan* plan, const uint32_t* d_c, uint32_t* d_U, size_t batch,
                        void* stream);

/*
 * Exact basis conversion (the u-corrected variant of App. B's fast conversion; the paper
 * prints only the fast one): d_out[b][j] = xbar mod p_j, where xbar is the centered CRT value
 * of d_in[b][.][c] in (-Q/2, Q/2), Q = prod q_i.  The multiple of Q that the fast conversion
 * adds is removed with v = round(sum_i [a_i qhat_i^-1]_{q_i} / q_i), estimated as a 128-bit
 * fixed-point sum with weights round(2^k / q_i), k = 63 + floor(log2 min q_i), so its error
 * is below eps = L max(q_i) 2^-(k+1) of Q (2^-57 for up to 64 sources of 28 bits): the result
 * is exact unless |xbar| lies within eps Q of Q/2 (then it may be the other representative's
 * residue).  Same layouts, plan and overlap rule as hefx_basis_convert; CUDA cores.
 */
hefx_status hefx_basis_convert_exact(hefx_ctx* ctx, const hefx_bconv_plan* plan, const uint32_t* d_in,
                                     uint32_t* d_out, size_t batch, void* stream);

/*
 * z = x o y mod q per limb (VecModMul of Table "HE operator -> AI operator"), elementwise over
 * [batch][nlimbs][N]; any of the buffers may alias.  Errors as for hefx_ntt_fwd.
 */
hefx_status hefx_vec_mod_mul(hefx_ctx* ctx, const hefx_params* params, const uint32_t* d_x, const uint32_t* d_y,
                             uint32_t* d_z, size_t batch, void* stream);

/*
 * z = x + y mod q per limb (VecModAdd, App. A), elementwise over [batch][nlimbs][N]; any of
 * the buffers may alias.  Errors as for hefx_ntt_fwd.
 */
hefx_status hefx_vec_mod_add(hefx_ctx* ctx, const hefx_params* params, const uint32_t* d_x, const uint32_t* d_y,
                             uint32_t* d_z, size_t batch, void* stream);

/*
 * Key-switching inner product of hybrid key switching with dnum digits (the HE-Mult /
 * Relin. measured in Sec. V-A and V-C, "Effects of Security Parameters"; App. A builds it
 * from VecModMul and VecModAdd): for each of `batch` inputs,
 *   d_out[b][k][l] = sum_{j < dnum} d_digits[b][j][l] o d_evk[j][k][l]  mod q_l,  k = 0, 1,
 * elementwise over the params' nlimbs limbs (the key-switching basis Q u P) in evaluation
 * form.  Layouts: d_digits [batch][dnum][nlimbs][N], d_evk [dnum][2][nlimbs][N] (shared by
 * the batch), d_out [batch][2][nlimbs][N]; inputs canonical.  d_out must not overlap an
 * input.  Errors: as for hefx_ntt_fwd, and EINVAL for dnum outside [1, 64] or overlap.
 * The paper keeps evaluation keys out of BAT (App. "Applying BAT to Preknown Parameters":
 * the dnum-long reduction is too short for a matrix engine); this runs on the CUDA cores.
 */
hefx_status hefx_key_inner_product(hefx_ctx* ctx, const hefx_params* params, const uint32_t* d_digits,
                                   const uint32_t* d_evk, uint32_t* d_out, uint32_t dnum, size_t batch, void* stream);

/*
 * ModDown of hybrid key switching (Sec. V-C; the formula is textbook RNS-CKKS, which the
 * paper cites but does not print): with `plan` a basis conversion from the special primes
 * P = p_0..p_{K-1} (its sources) to the ciphertext primes q_0..q_{L-1} (its targets),
 *   d_out[b][j] = (x[b][j] - BConv_{P->Q}(x[b][L..L+K-1])_j) * P^-1  mod q_j,   j < L,
 * where d_x is [batch][L + K][N] in coefficient form (the L ciphertext limbs, then the K
 * special limbs) and d_out is [batch][L][N].  The conversion is the fast one of
 * hefx_basis_convert, so the result represents floor(X / P) - u, 0 <= u < K, for the
 * integer X that d_x represents.  d_out must not overlap d_x.  Runs on the CUDA cores.
 * Errors: EINVAL for a null, foreign or misaligned argument or overlap.
 */
hefx_status hefx_mod_down(hefx_ctx* ctx, const hefx_bconv_plan* plan, const uint32_t* d_x, uint32_t* d_out,
                          size_t batch, void* stream);

/*
 * Rescale by the last prime of the parameter set (the HE operator Rescale of Sec. V-A;
 * textbook RNS-CKKS): for params over q_0..q_{L-1} (L >= 2), d_x [batch][L][N] and d_out
 * [batch][L-1][N], both in coefficient form,
 *   d_out[b][i] = (x[b][i] - (x[b][L-1] mod q_i)) * q_{L-1}^-1  mod q_i,   i < L - 1,
 * i.e. floor(X / q_{L-1}) for the integer X that d_x represents.  d_out may equal d_x when
 * batch == 1 (the result then occupies the first L - 1 rows); otherwise it must not overlap.
 * Errors: as for hefx_ntt_fwd, and EINVAL for L < 2 or overlap.
 */
hefx_status hefx_rescale(hefx_ctx* ctx, const hefx_params* params, const uint32_t* d_x, uint32_t* d_out,
                         size_t batch, void* stream);

/*
 * NTT(Rescale(x)): the rescaled polynomial in evaluation form over q_0 .. q_{L-2}, from x in
 * coefficient form over the params' L limbs -- hefx_rescale followed by the forward NTT of
 * its L - 1 limbs, with identical results.  For N >= 2^14 one launch: the transform's first
 * (cross-CTA) pass reads limb i and the last limb of the same polynomial and rescales on the
 * way in, so the rescaled polynomial never goes to memory; the limb tables of q_0 .. q_{L-2}
 * are the params' own.  Smaller N run the two steps (d_out is the workspace).  Layouts: d_x
 * [batch][L][N], d_out [batch][L - 1][N]; d_out must not overlap d_x.  Errors: as for
 * hefx_ntt_fwd; EINVAL for L < 2 or overlap; EUNSUPPORTED when the params' NTT reduction is
 * not the default (Shoup).
 */
hefx_status hefx_rescale_ntt(hefx_ctx* ctx, const hefx_params* params, const uint32_t* d_x, uint32_t* d_out,
                             size_t batch, void* stream);

/*
 * Tensor product of two ciphertexts (a0, a1), (b0, b1) in evaluation (NTT) form, the first
 * step of HE-Mult (Sec. III; App. A: HE-Mult is built from NTT, INTT, BConv, VecModMul and
 * VecModAdd): d0 = a0 o b0, d1 = a0 o b1 + a1 o b0, d2 = a1 o b1 mod q, elementwise over
 * [batch][nlimbs][N].  d_d2 may be null: d2 is then not written (a caller that only needs
 * INTT(d2) takes it from hefx_ntt_inv_hadamard(a1, b1)).  Outputs must not alias inputs.
 * Errors as for hefx_ntt_fwd.
 */
hefx_status hefx_tensor_product(hefx_ctx* ctx, const hefx_params* params, const uint32_t* d_a0, const uint32_t* d_a1,
                                const uint32_t* d_b0, const uint32_t* d_b1, uint32_t* d_d0, uint32_t* d_d1,
                                uint32_t* d_d2, size_t batch, void* stream);

/*
 * d_out = INTT(d_x o d_y) over the params' limbs (the inverse NTT of a Hadamard product, as in
 * the last step of hefx_poly_mul): the CUDA-core inverse transform multiplies the two inputs
 * (lazy Montgomery products, 2^32 folded into the final scale) as it loads them, with the same
 * results as hefx_vec_mod_mul then hefx_ntt_inv.  Layouts [batch][nlimbs][N] evaluation form
 * in, coefficient form out; d_out must not overlap an input (EINVAL).  Errors as for
 * hefx_ntt_fwd; EUNSUPPORTED when the params' NTT reduction is not the default (Shoup).
 */
hefx_status hefx_ntt_inv_hadamard(hefx_ctx* ctx, const hefx_params* params, const uint32_t* d_x, const uint32_t* d_y,
                                  uint32_t* d_out, size_t batch, void* stream);

/*
 * The HE-Mult front half of one ciphertext pair as one call (Sec. III HE-Mult, built from
 * NTT, INTT, BConv and VecModMul as in App. A): for ciphertexts (a0, a1), (b0, b1) over the
 * L limbs of `pq` in evaluation form and keys (k0, k1) over Q u P,
 *   d0 = a0 o b0, d1 = a0 o b1 + a1 o b0, d2 = a1 o b1,
 *   p = NTT_P(BConv_{Q->P}(INTT_Q(d2))),  e_k = (d2 o kq_k | p o kp_k),  k = 0, 1.
 * The plan records (does not own) the Q and P parameter sets, a conversion plan from Q's
 * primes to P's, and the key buffers kq_k [L][N], kp_k [K][N] (device, evaluation form).
 * Errors (create): EINVAL for null or foreign arguments, mismatched sizes, primes or N.
 */
typedef struct hefx_mult_plan hefx_mult_plan;
hefx_status hefx_mult_plan_create(hefx_ctx* ctx, const hefx_params* pq, const hefx_params* pp,
                                  const hefx_bconv_plan* bc, const uint32_t* d_kq0, const uint32_t* d_kq1,
                                  const uint32_t* d_kp0, const uint32_t* d_kp1, hefx_mult_plan** out);
void hefx_mult_plan_destroy(hefx_mult_plan* plan);

/*
 * Runs the front half on `stream`: d_in = [a0, a1, b0, b1], each [L][N]; d_out = [d0, d1,
 * e0 (Q part), e1 (Q part), e0 (P part), e1 (P part)], [4L + 2K][N] contiguous (one copy reads
 * every result); d_work [2L + K][N] holds d2, INTT(d2) and p.  The three must not overlap.
 * CUDA-core transforms; the conversion takes the path HEFX_PATH_AUTO picks for one polynomial
 * (see hefx_basis_convert); each pair of key products is one launch.
 * Errors: EINVAL for null, foreign, misaligned or overlapping buffers; ECUDA.
 */
hefx_status hefx_mult_front(hefx_ctx* ctx, const hefx_mult_plan* plan, const uint32_t* d_in, uint32_t* d_out,
                            uint32_t* d_work, void* stream);

/*
 * hefx_mult_front with host buffers: copies a0, a1, b0, b1 (host, [L][N] each; pinned memory
 * lets the copies overlap other work) into d_buf, runs the front half and copies the outputs
 * ([4L + 2K][N], layout of hefx_mult_front's d_out) back into h_out, all on `stream`.  When the
 * four inputs are equally spaced in host memory (h_a1 - h_a0 == h_b0 - h_a1 == h_b1 - h_b0 >=
 * L N words) they are uploaded as one pitched copy, else as four.  d_buf is device memory of
 * [10L + 3K][N] words (inputs, outputs, workspace).  Errors as above.
 */
hefx_status hefx_mult_front_host(hefx_ctx* ctx, const hefx_mult_plan* plan, const uint32_t* h_a0,
                                 const uint32_t* h_a1, const uint32_t* h_b0, const uint32_t* h_b1, uint32_t* h_out,
                                 uint32_t* d_buf, void* stream);

/*
 * Several serving requests of one ring degree in shared launches (the batching of the
 * serving loop; the paper's batching study is Sec. V-B3).  Each request r is a front half as
 * in hefx_mult_front_host: plan plans[r] (requests may differ in limb count L_r, i.e. in Q
 * parameter set, conversion plan and keys, but share N and the P parameter set), host inputs
 * h_a0[r] .. h_b1[r], host output h_out[r], device buffer d_buf[r] of [10 L_r + 3K][N] words.
 * Per request the inputs are uploaded and the outputs read back; every stage runs ONCE over
 * all requests' rows: the tensor product and the key products as row-list elementwise
 * launches, INTT(d2) and NTT over P as row-list transforms, BConv_{Q->P} as one launch with a
 * block row per request (CUDA-core conversion).  Results equal hefx_mult_front_host's, bit
 * for bit.  The batch object owns a ring of descriptor slots (pinned host + device): create
 * it once with the largest count and limb count to serve; a call reuses a slot only after the
 * launches that read it have completed.  All on `stream`.
 * Errors: EINVAL (null or foreign arguments, count or limbs above the object's, mixed N or P,
 * misaligned buffers), EUNSUPPORTED (more than 64 special limbs), ENOMEM (create), ECUDA.
 */
typedef struct hefx_mult_batch hefx_mult_batch;
hefx_status hefx_mult_batch_create(hefx_ctx* ctx, uint32_t max_requests, uint32_t max_limbs, hefx_mult_batch** out);
void hefx_mult_batch_destroy(hefx_mult_batch* batch);
hefx_status hefx_mult_front_batch_host(hefx_ctx* ctx, hefx_mult_batch* batch, const hefx_mult_plan* const* plans,
                                       uint32_t count, const uint32_t* const* h_a0, const uint32_t* const* h_a1,
                                       const uint32_t* const* h_b0, const uint32_t* const* h_b1,
                                       uint32_t* const* h_out, uint32_t* const* d_buf, void* stream);

/*
 * The same batched front half on device-resident operands (the serving loop's resident mode:
 * ciphertexts and keys stay in HBM between operations, nothing crosses the host link): request
 * r reads d_a0[r] .. d_b1[r] ([L_r][N] each, device) and writes d_out[r] ([4 L_r + 2K][N], the
 * layout of hefx_mult_front's d_out) using d_work[r] ([2 L_r + K][N]) as workspace.  A
 * request's output and workspace must not overlap any of its buffers; distinct requests must
 * not share outputs or workspaces.  Results equal hefx_mult_front's, bit for bit.  All on
 * `stream`.  Errors as for hefx_mult_front_batch_host.
 */
hefx_status hefx_mult_front_batch(hefx_ctx* ctx, hefx_mult_batch* batch, const hefx_mult_plan* const* plans,
                                  uint32_t count, const uint32_t* const* d_a0, const uint32_t* const* d_a1,
                                  const uint32_t* const* d_b0, const uint32_t* const* d_b1, uint32_t* const* d_out,
                                  uint32_t* const* d_work, void* stream);

/*
 * Native serving loop (the request loop of the build's serving pattern; continuous batching of
 * HE-Mult front-half requests on device-resident ciphertexts).  Runs in real time on the
 * calling host thread until every request is done or rejected:
 *  - request i arrives reqs[i].arrival_s seconds after the call starts (sorted by arrival);
 *    one needing more than budget_bytes is rejected;
 *  - admission is FIFO (head-of-line blocking) while the bytes of the admitted requests fit
 *    budget_bytes and a result slot is free;
 *  - the requests admitted in one pass are grouped by ring degree and P parameter set and
 *    each group of at most max_group runs as one hefx_mult_front_batch on the next of the
 *    streams (round-robin) with the request's result slot as output (slot_out[k]:
 *    [4L + 2K][N] words, slot_work[k]: [2L + K][N], for the largest request served);
 *  - a group completes with an event recorded after its launches; its requests' slots and
 *    bytes are then released.
 * out[i] receives the admission and completion times (seconds from the start), the status and
 * the slot that holds the results (valid until the slot is reused by a later request).  The
 * caller owns every buffer and stream.  Errors: EINVAL (null or foreign arguments, unsorted
 * arrivals), ECUDA (the run stops after waiting for the launched groups).
 */
typedef enum { HEFX_SERVE_PENDING = 0, HEFX_SERVE_RUNNING = 1, HEFX_SERVE_DONE = 2, HEFX_SERVE_REJECTED = 3 } hefx_serve_status;
typedef struct {
    double arrival_s;
    const hefx_mult_plan* plan;
    const uint32_t* d_a0;
    const uint32_t* d_a1;
    const uint32_t* d_b0;
    const uint32_t* d_b1;
    uint64_t bytes;  /* device bytes charged against the budget while the request runs */
} hefx_serve_request;
typedef struct {
    double admitted_s;
    double completed_s;
    int32_t status; /* hefx_serve_status */
    uint32_t slot;
} hefx_serve_result;
typedef struct {
    uint64_t max_active;
    uint64_t memory_high_water_bytes;
    uint64_t groups;
} hefx_serve_stats;
typedef struct {
    uint32_t nstreams;
    void* const* streams;
    uint32_t nslots;
    uint32_t* const* slot_out;
    uint32_t* const* slot_work;
    uint64_t budget_bytes;
    uint32_t max_group;
    hefx_serve_stats* stats; /* optional */
} hefx_serve_config;
hefx_status hefx_serve_run(hefx_ctx* ctx, hefx_mult_batch* batch, const hefx_serve_request* reqs, size_t n,
                           const hefx_serve_config* cfg, hefx_serve_result* out);

/*
 * Batched polynomial products of uneven shape (the batching pattern of the build; the
 * paper's batching study is Sec. V-B3, "TPUs favor large batch").  Each job multiplies two
 * polynomials of ring degree N = 2^params->log2n over the first `nlimbs` primes of
 * `params` (limb i uses prime i), data laid out [nlimbs][N] in natural coefficient order.
 * d_c may alias d_a and/or d_b; distinct jobs must not overlap.
 */
typedef struct {
    const hefx_params* params;
    uint32_t nlimbs;
    const uint32_t* d_a;
    const uint32_t* d_b;
    uint32_t* d_c;
} hefx_job;

typedef struct hefx_batch_plan hefx_batch_plan;

/*
 * Builds the device work lists of a batch once: every limb of every job becomes one row
 * descriptor (carrying its parameter set's tables).  When every job's ring degree is in
 * [2^10, 2^16] and every modulus is below 2^28, the rows are cut into cluster tasks of 2^16
 * elements of one ring degree (one row of 2^16, two of 2^15, four of 2^14, or 8 CTA-sized
 * groups of smaller rows; largest ring degree first) and the whole batch runs as ONE launch
 * of the fused batch kernel; otherwise jobs are grouped by parameter set and each size class
 * takes two row-list launches.  The buffers named by the jobs must stay valid for the plan's
 * lifetime.  path: AUTO or CUDACORE (the CUDA-core kernels); TENSOR gives EUNSUPPORTED.
 * Errors: EINVAL (null/misaligned pointer, nlimbs out of range, params of another context),
 * EUNSUPPORTED, ENOMEM.
 */
hefx_status hefx_batch_plan_create(hefx_ctx* ctx, const hefx_job* jobs, size_t njobs, hefx_path path,
                                   hefx_batch_plan** out);
void hefx_batch_plan_destroy(hefx_batch_plan* plan);

/*
 * Kernel launches one hefx_batch_polymul of the plan makes (1 for the fused form).
 */
uint32_t hefx_batch_plan_launches(const hefx_batch_plan* plan);

/*
 * Runs every job of the plan: c = INTT(NTT(a) o NTT(b)) per limb (INTT(NTT(a) o NTT(a)) when
 * a == b); in the fused form one launch in which each cluster computes NTT(a) into c and then
 * INTT(NTT(b) o c) into c for its task's rows, otherwise per size class one launch of each
 * half.  On a non-default stream that is not already
 * being captured, the first call captures these launches into a CUDA graph and every call
 * replays it (one graph launch per batch); on the legacy default stream, or inside a
 * caller's own capture, the kernels are launched directly.  Errors: EINVAL, ECUDA.
 */
hefx_status hefx_batch_polymul(hefx_ctx* ctx, hefx_batch_plan* plan, void* stream);

/*
 * Waits for `stream`, then reports whether a bounded device-side wait of the tensor-path
 * kernels launched with `params` expired since the last check (HEFX_ETIMEOUT; the results of
 * those calls are invalid) and clears that record.  The tcgen05 pipelines wait on mbarriers
 * with a time limit instead of spinning forever, so a failure ends the kernel with a
 * recorded code rather than a hung device.  Errors: EINVAL, ECUDA, ETIMEOUT.
 */
hefx_status hefx_stream_check(hefx_ctx* ctx, const hefx_params* params, void* stream);

/*
 * Check of the failure-detection path (no counterpart in the paper: a property of this
 * library's kernels).  Every wait of the tensor-core and TMA pipelines is bounded: when a
 * copy or an MMA it waits for does not arrive within the limit, the waiting thread records
 * an error code in a device flag, the kernel releases what it holds (TMEM) and returns, and
 * hefx_stream_check reports HEFX_ETIMEOUT instead of the device hanging.  This call runs that
 * same bounded wait in a one-warp kernel that holds TMEM while it waits on an mbarrier:
 *  - arrive != 0: the kernel arrives on the barrier first; the wait succeeds and the next
 *    hefx_stream_check(ctx, params, stream) returns HEFX_OK;
 *  - arrive == 0: nothing ever arrives; the wait gives up after limit_ns nanoseconds, the
 *    code is recorded in params' error flag and the next hefx_stream_check returns
 *    HEFX_ETIMEOUT (and clears the flag).  The context stays usable.
 * limit_ns at most 2e9 (the pipelines' own limit), else HEFX_EINVAL.  Asynchronous on stream.
 * Errors: EINVAL, ECUDA.
 */
hefx_status hefx_wait_check(hefx_ctx* ctx, const hefx_params* params, uint64_t limit_ns, int arrive, void* stream);

#ifdef __cplusplus
}
#endif

#endif /* HEFX_H */
