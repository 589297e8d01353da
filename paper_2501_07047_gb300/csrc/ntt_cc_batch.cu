// Fused batch kernel: the whole uneven batch of polynomial products (jobs of ring degrees
// 2^10 .. 2^16 with their own limb counts) in one launch.  Each cluster of 8 CTAs (128 threads,
// 2^13 elements of shared memory each) takes one task of 2^16 elements of one ring degree:
// one row of 2^16, two rows of 2^15, four of 2^14 (the row's CTAs exchange data through
// distributed shared memory within their part of the cluster), or 8 CTA-sized groups of
// smaller rows.  A task runs both halves of its rows' products back to back: c = NTT(a), then
// c = INTT(NTT(b) o c) (or INTT(c o c) for squares), the same two transforms the per-size
// launches run (App. A radix-2 NTT; Table "HE operator -> AI operator": NTT, Hadamard, INTT).
// Row descriptors carry each row's own constant and twiddle tables, so tasks of every ring
// degree share the launch, and the hardware schedules the clusters as they free up.
#include <cstring>

#include "ntt_cc_impl.cuh"

namespace hefx {
namespace cc {

namespace {

constexpr int kBatchMinLog = 10, kBatchMaxLog = 16;

template <int LOGN, int F>
__device__ __forceinline__ void batch_task(uint32_t* sm, const BatchTask& t, uint32_t rank, const KArgs& a,
                                           uint32_t off2, uint64_t* bar, uint32_t& ph) {
    using C = Cfg<LOGN, F>;
    static_assert(C::unified && C::threads == 128 && C::elems == 8192, "one 2^13-element CTA per cluster rank");
    Seg sg;
    if constexpr (C::split) {
        const uint32_t sub = rank / C::P;  // which row of the task (the plan fills split tasks)
        sg.row0 = t.row0 + sub;
        sg.part = rank % C::P;
        sg.nrows = 1;
        sg.rbase = sub * C::P;
    } else {
        const uint32_t first = t.row0 + rank * C::rows, end = t.row0 + t.nrows;
        sg.row0 = first;
        sg.part = 0;
        sg.nrows = first < end ? (int)min((uint32_t)C::rows, end - first) : 0;
        sg.rbase = 0;
    }
    sg.gbase = sg.part * C::m;
    if (C::split || sg.nrows > 0) run_task<LOGN, MODE_FWD, F>(sm, sg, a, bar, ph);
    // the second half reads c (written above by this CTA, for its own part of each row) and,
    // in split rows, writes into the peers' shared memory: every CTA of the cluster is done
    // with the first half before it starts
    __threadfence_block();
    if constexpr (C::split) cg::this_cluster().sync();
    else __syncthreads();
    Seg s2 = sg;
    s2.row0 += off2;
    if (C::split || sg.nrows > 0) {
        if (t.mode == MODE_HAD_INV) run_task<LOGN, MODE_HAD_INV, F>(sm, s2, a, bar, ph);
        else run_task<LOGN, MODE_FWD_HAD_INV, F>(sm, s2, a, bar, ph);
    }
}

template <int F>
__global__ void __launch_bounds__(128, 5) ntt_cc_batch_kernel(const __grid_constant__ KArgs a,
                                                               const BatchTask* __restrict__ tasks, uint32_t off2) {
    extern __shared__ __align__(16) uint32_t sm[];
    __shared__ uint64_t bar;  // unused: row lists take no TMA copies
    uint32_t ph = 0, rank;
    asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(rank));
    griddep_wait();
    const BatchTask t = tasks[blockIdx.x / 8];
    switch (t.logn) {
        case 16: batch_task<16, F>(sm, t, rank, a, off2, &bar, ph); break;
        case 15: batch_task<15, F>(sm, t, rank, a, off2, &bar, ph); break;
        case 14: batch_task<14, F>(sm, t, rank, a, off2, &bar, ph); break;
        case 13: batch_task<13, F>(sm, t, rank, a, off2, &bar, ph); break;
        case 12: batch_task<12, F>(sm, t, rank, a, off2, &bar, ph); break;
        case 11: batch_task<11, F>(sm, t, rank, a, off2, &bar, ph); break;
        default: batch_task<10, F>(sm, t, rank, a, off2, &bar, ph); break;
    }
}

}  // namespace

}  // namespace cc

bool ntt_cc_batch_supported(uint32_t log2n, bool lazy) {
    return lazy && (int)log2n >= cc::kBatchMinLog && (int)log2n <= cc::kBatchMaxLog;
}

uint32_t ntt_cc_batch_rows_per_task(uint32_t log2n) {
    return log2n >= 13 ? 1u << (16 - log2n) : 8u << (13 - log2n);
}

// One launch: one cluster of 8 CTAs per task; rows [0, off2) are the first halves' descriptors
// and rows [off2, 2 off2) the second halves'.
cudaError_t launch_ntt_cc_batch(const RowDesc* d_rows, const BatchTask* d_tasks, uint32_t ntasks, uint32_t off2,
                                uint32_t* err, cudaStream_t stream) {
    if (ntasks == 0) return cudaSuccess;
    cc::KArgs a;
    memset(&a, 0, sizeof a);
    a.err = err;
    a.desc = d_rows;
    a.rows = 2 * off2;
    a.L = 1;
    cudaLaunchConfig_t cfg = {};
    cudaLaunchAttribute attr[2];
    cfg.gridDim = dim3(8 * ntasks);
    cfg.blockDim = dim3(128);
    cfg.dynamicSmemBytes = 8192 * 4;
    cfg.stream = stream;
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    attr[1].id = cudaLaunchAttributeClusterDimension;
    attr[1].val.clusterDim.x = 8;
    attr[1].val.clusterDim.y = 1;
    attr[1].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 2;
    return cudaLaunchKernelEx(&cfg, cc::ntt_cc_batch_kernel<3 | 16>, a, d_tasks, off2);
}

}  // namespace hefx
