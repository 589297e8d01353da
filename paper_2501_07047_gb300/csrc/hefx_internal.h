// Internal types shared by the hefx host API and its kernels (not part of the C ABI).
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>

#include <cstdint>
#include <mutex>
#include <string>
#include <vector>

#include "../../include/hefx.h"

namespace hefx {

typedef int NttModeTag;  // an NttMode value, stored by plans

// Per-limb constants of one parameter set, in device memory ([nlimbs] array).
struct LimbConst {
    uint32_t q;
    uint32_t qinv_neg;            // -q^-1 mod 2^32 (Montgomery REDC)
    uint32_t ninv, ninv_sh;       // N^-1 mod q and its Shoup companion
    uint32_t ninvw, ninvw_sh;     // N^-1 * psi^-brv_N(1): twiddle of the last Gentleman-Sande stage
    uint32_t ninvR, ninvR_sh;     // N^-1 * 2^32: undoes the 2^-32 of a Montgomery Hadamard product
    uint32_t ninvRw, ninvRw_sh;   // N^-1 * 2^32 * psi^-brv_N(1)
    uint32_t r2;                  // 2^64 mod q: two Montgomery products give a plain one
    uint32_t one_sh;              // floor(2^32 / q), Shoup companion of 1: any x < 2^32 -> [0, 2q)
    uint32_t rs_inv, rs_inv_sh;   // q_{L-1}^-1 mod q (Rescale by the set's last prime) and companion
    uint32_t bar_lo, bar_hi;      // floor(2^64 / q) (Barrett reduction variant)
    // 2q, 4q, 8q, read from memory by the NTT butterflies (the lazy offsets X - Y + c q): as
    // loaded values they stay in registers and each offset add is one three-input add,
    // where a multiple of q the compiler derives itself is recomputed with a shift-add
    uint32_t q2, q4, q8;
    uint32_t pad_[13];
};
static_assert(sizeof(LimbConst) == 128, "LimbConst is one 128-byte line");

// Number of stages in the CUDA-core NTT's smallest-stride register pass for N = 2^log2n.
// The twiddle entries of those stages are stored permuted (see hefx_params_create) so that
// the per-lane loads of that pass are coalesced.
inline constexpr int ntt_cc_small_radix(int log2n) {
    return (log2n >= 16 ? log2n - 1 : log2n) < 5 ? (log2n >= 16 ? log2n - 1 : log2n) : 5;
}

// One row (limb of one polynomial) of a batched job: where its operands live and which limb
// of the parameter set's basis it is reduced by.
struct RowDesc {
    const uint32_t* in;
    const uint32_t* had;
    uint32_t* out;
    const LimbConst* lc;  // the row's limb constants (its parameter set's table, limb resolved)
    const uint2* twf;     // the row's forward twiddles (N entries)
    const uint2* twi;     // the row's inverse twiddles (N entries)
    uint32_t limb;
    uint32_t pad[3];
};
static_assert(sizeof(RowDesc) == 64, "RowDesc is one 64-byte line");

// One conversion of a list launch (bconv.cu, serving batches): plan constants (a plan's
// d_const), one polynomial's source limbs and its output limbs.
struct BcListEntry {
    const void* c;
    const uint32_t* in;
    uint32_t* out;
};

// One cluster task of the fused batch kernel (ntt_cc_batch.cu): nrows rows of ring degree
// 2^logn whose first-half descriptors start at row0 (second halves at row0 + the plan's offset).
struct BatchTask {
    uint32_t logn;
    uint32_t mode;  // second half: MODE_FWD_HAD_INV, or MODE_HAD_INV for squares
    uint32_t row0;
    uint32_t nrows;
};

// Device tables of the tensor-core (matrix) NTT for one parameter set: the single-pass GEMMs
// of ntt_tc.cu (used by the no-allocation product) and the pipelined GEMMs of ntt_tc2.cu.
struct TensorTables;
struct Tc2Tables;

}  // namespace hefx

struct hefx_ctx {
    int device = 0;
    int sm_count = 0;
    std::string last_error;
    std::mutex mu;
    // co-resident clusters of the N = 2^16 CUDA-core transform, [inverse][28-bit moduli]
    // (-1: not queried yet)
    int cc16_clusters[2][2] = {{-1, -1}, {-1, -1}};
};

struct hefx_params {
    hefx_ctx* ctx = nullptr;
    uint32_t log2n = 0;
    uint32_t n = 0;
    uint32_t nlimbs = 0;
    std::vector<uint32_t> primes;
    std::vector<uint32_t> psi;        // per limb
    uint32_t max_prime = 0;
    hefx::LimbConst* d_lc = nullptr;  // [nlimbs]
    uint2* d_tw_fwd = nullptr;        // [nlimbs][N]: (psi^brv_N(k), Shoup companion), k >= 1
    uint2* d_tw_inv = nullptr;        // [nlimbs][N]: (psi^-brv_N(k), Shoup companion)
    // N = 2^16 only: the same tables with the smallest-stride group-major part over 4 stages
    // (the two-pass CUDA-core transform, ntt_cc_2p.cu); null for other ring degrees
    uint2* d_tw2_fwd = nullptr;
    uint2* d_tw2_inv = nullptr;
    int cc_schedule = 0;              // hefx_cc_schedule of the contiguous CUDA-core transforms
    hefx::TensorTables* tc = nullptr; // built on first tensor-path use
    hefx::Tc2Tables* tc2 = nullptr;   // built on first tensor-path use
    std::mutex tc_mu;
    hefx_path tuned_path = HEFX_PATH_AUTO;
    uint32_t tc_log2r = 0;            // tensor-path split: log2 of the first factor (0: 2^floor(log2n / 2))
    uint32_t tc_log2r2 = 0;           // log2 of the second factor of a three-factor split (0: two factors)
    int tc_tile = 64;                 // tensor-path GEMM tile: outputs per tile (64 or 32)
    int red_ntt = 0;                  // hefx_reduction of the CUDA-core twiddle products
    int red_vec = 1;                  // hefx_reduction of VecModMul
    uint2* d_tw_fwd_mont = nullptr;   // Montgomery-form twiddles (w 2^32 mod q), built on demand
    uint2* d_tw_inv_mont = nullptr;
    uint32_t* d_err_cc = nullptr;     // CUDA-core kernels' bounded-wait error flag
};

struct hefx_batch_plan {
    hefx_ctx* ctx = nullptr;
    struct Launch {
        const hefx_params* params;
        hefx::NttModeTag mode;
        size_t offset;  // first RowDesc of this launch in d_rows
        size_t nrows;
    };
    std::vector<Launch> launches;
    // fused form (every job's ring degree in [2^10, 2^16], 28-bit moduli): one launch of
    // ntasks cluster tasks over d_rows (first halves, then second halves at row off2)
    bool fused = false;
    void* d_tasks = nullptr;  // BatchTask array
    uint32_t ntasks = 0, off2 = 0;
    uint32_t* d_pad = nullptr;  // scratch rows that fill the last task of a split ring degree
    uint32_t* err = nullptr;
    void* d_rows = nullptr;  // RowDesc array
    size_t total_rows = 0;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    cudaStream_t graph_stream = nullptr;  // stream the graph was captured on
};

struct hefx_bconv_plan {
    hefx_ctx* ctx = nullptr;
    uint32_t log2n = 0;
    uint32_t L = 0, Lp = 0;
    std::vector<uint32_t> src, dst;
    void* d_const = nullptr;          // BConvConst (see bconv.cu)
    void* d_bat = nullptr;            // BAT digit matrix of step 2 (fp16), see bconv.cu
    uint32_t* d_err = nullptr;        // bounded-wait error flag of the pipelined kernels (0 = none)
};

// ModUp of hybrid key switching (bconv.cu): one plan for every digit of (Q, P, alpha).
struct hefx_modup_plan {
    hefx_ctx* ctx = nullptr;
    uint32_t log2n = 0;
    uint32_t L = 0, K = 0, alpha = 0, dnum = 0;
    std::vector<uint32_t> q, p;
    void* d_const = nullptr;  // dnum BConvConst
};

namespace hefx {

// Programmatic dependent launch: a kernel launched this way may start (set-up only) while the
// stream's preceding kernel drains; it runs griddep_wait() before its first access to memory
// that a preceding kernel writes or reads, which then waits for that kernel to complete.  No
// early trigger is issued anywhere, so a dependent launch starts only after every block of
// the preceding kernel has exited.  griddep_wait() is a no-op for a plain launch.
#ifdef __CUDACC__
__device__ __forceinline__ void griddep_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }


template <typename... Params, typename... Args>
cudaError_t launch_pdl(void (*kern)(Params...), dim3 grid, dim3 block, size_t smem, cudaStream_t s, Args... args) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    at[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, kern, args...);
}
#endif

// Kernel launchers (return a CUDA error code; the host API maps it to hefx_status).
// MODE_RS_FWD: NTT(Rescale(x)): the forward transform of q_0..q_{L-2} whose first pass reads
// limb i and the last limb of the same coefficient-form polynomial and rescales on the way in.
enum NttMode { MODE_FWD = 0, MODE_INV = 1, MODE_FWD_HAD_INV = 2, MODE_HAD_INV = 3, MODE_RS_FWD = 4 };

// Two-pass CUDA-core transform of contiguous N = 2^16 rows [batch][L][N] (forward or inverse;
// in may equal out).  cudaErrorNotSupported where ntt_cc_2p_supported is false.
bool ntt_cc_2p_supported(const hefx_params* p, NttMode mode);
cudaError_t launch_ntt_cc_2p(const hefx_params* p, NttMode mode, const uint32_t* in, uint32_t* out, size_t rows,
                             cudaStream_t stream);
cudaError_t launch_ntt_cc(const hefx_params* p, NttMode mode, const uint32_t* in, const uint32_t* had, uint32_t* out,
                          size_t rows, cudaStream_t stream);
// Elementwise products of the HE-Mult request (elementwise.cu).
cudaError_t launch_vec_mod_mul(const hefx_params* p, const uint32_t* x, const uint32_t* y, uint32_t* z, size_t rows,
                               cudaStream_t s);
// z0 = x o y0 and z1 = x o y1 in one pass (the default Montgomery reduction; else two launches).
cudaError_t launch_vec_mod_mul2(const hefx_params* p, const uint32_t* x, const uint32_t* y0, const uint32_t* y1,
                                uint32_t* z0, uint32_t* z1, size_t rows, cudaStream_t s);
// VecModMul with the BAT lazy reduction on the tensor cores (bat_lazy.cu); log2n >= 9.
cudaError_t launch_vec_mod_mul_bat(const hefx_params* p, const uint32_t* x, const uint32_t* y, uint32_t* z,
                                   size_t rows, cudaStream_t s);
cudaError_t launch_tensor_product(const hefx_params* p, const uint32_t* a0, const uint32_t* a1, const uint32_t* b0,
                                  const uint32_t* b1, uint32_t* d0, uint32_t* d1, uint32_t* d2, size_t rows,
                                  cudaStream_t s);

// Sets the kernel attributes of (N, mode) ahead of time (no launch), e.g. before a capture.
cudaError_t prepare_ntt_cc(const hefx_params* p, NttMode mode);
// Same kernels over an explicit list of rows (device array of RowDesc), persistent grid.
// out[b] (evaluation form over q_0..q_{L-2}) = NTT(Rescale(in[b])), in [batch][L][N] coefficient
// form over the params' L limbs: one fused launch where built (N >= 2^14, contiguous),
// else the rescale kernel then the forward transform.
cudaError_t launch_ntt_cc_rescale(const hefx_params* p, const uint32_t* in, uint32_t* out, size_t batch,
                                  cudaStream_t stream);
cudaError_t launch_ntt_cc_rows(const hefx_params* p, NttMode mode, const RowDesc* d_rows, size_t nrows,
                               cudaStream_t stream);

cudaError_t encode_input_map(const hefx_params* p, const uint32_t* in, size_t rows, CUtensorMap* map);
cudaError_t launch_ntt_cc_red(const hefx_params* p, NttMode mode, uint32_t* data, size_t rows, cudaStream_t stream);
cudaError_t make_mont_twiddles(const hefx_params* p, const uint2* tw, uint2* out);
cudaError_t launch_vec_mod_add(const hefx_params* p, const uint32_t* x, const uint32_t* y, uint32_t* z, size_t rows,
                               cudaStream_t s);
cudaError_t launch_key_inner_product(const hefx_params* p, const uint32_t* dig, const uint32_t* evk, uint32_t* out,
                                     uint32_t dnum, size_t batch, cudaStream_t s);
cudaError_t launch_rescale(const hefx_params* p, const uint32_t* x, uint32_t* out, size_t batch, cudaStream_t s);
cudaError_t launch_bconv_exact(const hefx_bconv_plan* plan, const uint32_t* in, uint32_t* out, size_t batch,
                               cudaStream_t stream);
cudaError_t launch_mod_down(const hefx_bconv_plan* plan, const uint32_t* x, uint32_t* out, size_t batch,
                            cudaStream_t stream);
cudaError_t launch_bconv_cc(const hefx_bconv_plan* plan, const uint32_t* in, uint32_t* out, size_t batch,
                            cudaStream_t stream);
// The plain conversion with TMA-fed tiles (bconv_cc_tma.cu): L <= 48 sources, N >= 2^8;
// cudaErrorNotSupported otherwise.
cudaError_t launch_bconv_cc_tma(const hefx_bconv_plan* plan, const uint32_t* in, uint32_t* out, size_t batch,
                                uint32_t* err, cudaStream_t stream);
cudaError_t bconv_plan_upload(hefx_bconv_plan* plan);
cudaError_t modup_plan_upload(hefx_modup_plan* plan);
// U[b][j] = ModUp digit j of c[b] ([batch][L][N] -> [batch][dnum][L + K][N], coefficient form)
cudaError_t launch_mod_up(const hefx_modup_plan* plan, const uint32_t* c, uint32_t* U, size_t batch,
                          cudaStream_t stream);
void bconv_plan_free(hefx_bconv_plan* plan);

// Tensor-core path (ntt_tc.cu / bconv_tc.cu).
// The pipelined tensor NTT (ntt_tc2.cu) runs N = 2^14 .. 2^16 for every modulus below 2^30
// (8-bit digits above 2^28); the single-pass form (ntt_tc.cu, the no-allocation product)
// needs moduli below 2^28.
bool tc_supported(const hefx_params* p);
bool tc_narrow(const hefx_params* p);
inline bool tc2_wide(const hefx_params* p) { return p->max_prime >= (1u << 28); }
cudaError_t tc_prepare(hefx_params* p);
void tc_free(hefx_params* p);
cudaError_t tc_check(const hefx_params* p, cudaStream_t stream, uint32_t* code);
size_t noalloc_scratch_words();
cudaError_t launch_wait_check(uint32_t* err, uint64_t limit_ns, int arrive, cudaStream_t stream);
// Read access to a serving plan's fields (hefx_api.cu) for the batched request (mult_batch.cu).
struct MultPlanView {
    hefx_ctx* ctx;
    const hefx_params* pq;
    const hefx_params* pp;
    const hefx_bconv_plan* bc;
    const uint32_t* kq[2];
    const uint32_t* kp[2];
};
bool mult_plan_view(const hefx_mult_plan* plan, MultPlanView* out);
// The batched front half on device pointers (mult_batch.cu; hefx_mult_front_batch's body):
// inputs[i][r] request r's input i, d_out[r] its outputs, d_work[r] its workspace.
hefx_status mult_front_batch_dev(hefx_ctx* ctx, hefx_mult_batch* mb, const hefx_mult_plan* const* plans,
                                 uint32_t count, const uint32_t* const* const inputs[4], uint32_t* const* d_out,
                                 uint32_t* const* d_work, cudaStream_t s);
cudaError_t launch_bconv_cc_list(const BcListEntry* d_list, uint32_t count, uint32_t log2n, uint32_t lp_max,
                                 cudaStream_t stream);
// Fused batch kernel (ntt_cc_batch.cu).
bool ntt_cc_batch_supported(uint32_t log2n, bool lazy);
uint32_t ntt_cc_batch_rows_per_task(uint32_t log2n);
cudaError_t launch_ntt_cc_batch(const RowDesc* d_rows, const BatchTask* d_tasks, uint32_t ntasks, uint32_t off2,
                                uint32_t* err, cudaStream_t stream);
cudaError_t tc2_prepare(hefx_params* p);
void tc2_free(hefx_params* p);
uint32_t* tc2_err(const hefx_params* p);
cudaError_t tc2_forward(hefx_params* p, const uint32_t* in, uint32_t* out, int mul, const uint32_t* had, size_t batch,
                        cudaStream_t s);
cudaError_t tc2_inverse(hefx_params* p, const uint32_t* in, uint32_t* out, size_t batch, cudaStream_t s);
cudaError_t tc2_polymul(hefx_params* p, const uint32_t* a, const uint32_t* b, uint32_t* c, size_t batch,
                        cudaStream_t s);
cudaError_t polymul_tc_noalloc(const hefx_params* p, const uint32_t* a, const uint32_t* b, uint32_t* c, size_t batch,
                               cudaStream_t stream);
cudaError_t launch_bconv_tc(const hefx_bconv_plan* plan, const uint32_t* in, uint32_t* out, size_t batch,
                            cudaStream_t stream);

}  // namespace hefx
