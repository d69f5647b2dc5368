// k_dfb.cu -- directional filter bank stages (§2.1), fused tile kernels.
//
// Every stage is a two-channel fan filter bank in ladder form (see
// ct_engine.cu for the lattice reading): one pass over the target coset, one
// over the other, each sample becoming alpha*self + gamma*(NT x NT stencil of
// the other coset) with weights bt[a]*bt[b], bt the fan taps of the NT-tap
// prototype (NT = 4: (-1,-9,9,1)/16; 6 and 8: the longer Lagrange half-band
// prototypes).  Both kernels are templates on NT; a pass reaches R = NT - 1
// samples.
//
// k_dfb_a: stages 1 and 2 of a detail image in 64 x 64 tiles.  The tile and
//   a 4R-sample halo (R per pass) sit in shared memory as the image's four
//   polyphase planes (the stage-2 channels), so every pass reads unit-stride
//   rows without bank conflicts; the tap tables are compile-time constants;
//   the four passes run in place; the planes are written to the channel
//   arrays, or read from them in the synthesis direction.
// k_dfb_b: one stage s >= 3 of a channel array (a split into even / odd
//   rows).  Rows are staged in shared memory SHEARED by i*q + r columns (q
//   the parent row, r the tile row), which turns the slope-i stencil (row
//   offset a, column offset -i*a + (b-a)/2) into one NT x NT rectangle for
//   every i; it is evaluated separably, an NT-tap sum across rows of NT-tap
//   row sums.  A thread takes a quad of 4 adjacent targets and walks down
//   its rows: consecutive targets share all but one row sum, so the row sums
//   live in registers, and every shared-memory access is a 16-byte vector.
//   Both passes of the stage run in one launch on a 16-row tile, 128 columns
//   staged with an R-row / R-column halo.
//
// Both directions compute in single precision: the filter-bank weights are
// dyadic and alpha, gamma powers of two, and the inverse's error is dominated
// by the Laplacian-pyramid synthesis, which is compensated (k_lp.cu).
#include <mutex>

#include "dfb_tile.cuh"

namespace cvc {

// stages 1 + 2, one block per (job, tile); blocks of streams that take no part return
template <bool SYN, int NT>
__global__ void __launch_bounds__(256) k_dfb_a(const DfbAJob* __restrict__ jobs, const int* __restrict__ block_job,
                                               Bases B, PassParams pp) {
    extern __shared__ __align__(16) float smem_a[];
    const DfbAJob& J = jobs[block_job[blockIdx.x]];
    if (job_idle(B, J.stream)) return;
    dfb_a_tile<SYN, NT>(J, blockIdx.x - J.first_block, B, pp, smem_a);
}

// one row-split stage, one block of TH threads per (job, tile); FO: the first target coset is odd
template <bool SYN, int NT, bool FO, int TH>
__global__ void __launch_bounds__(TH, TH == DFBB_THREADS ? (NT == 8 ? 6 : 8) : (NT == 8 ? 3 : 4))
    k_dfb_b(const DfbBJob* __restrict__ jobs, const int* __restrict__ block_job, Bases B, PassParams pp) {
    using G = BGeo<NT>;
    __shared__ __align__(16) float sE[G::SMB];
    __shared__ __align__(16) float sO[G::SMB];
    const DfbBJob& J = jobs[block_job[blockIdx.x]];
    if (job_idle(B, J.stream)) return;
    dfb_b_tile<SYN, NT, FO, false, TH>(J, blockIdx.x - J.first_block, B, pp, sE, sO);
}

// ============================================================ launches
cudaError_t dfb_prepare() {
    // the stage-1+2 tiles of the longer prototypes need more than 48 KB of dynamic shared memory
    static std::once_flag once;
    static cudaError_t status = cudaSuccess;
    std::call_once(once, [] {
        const int s6 = AGeo<6>::SMEM, s8 = AGeo<8>::SMEM;
        const cudaFuncAttribute a = cudaFuncAttributeMaxDynamicSharedMemorySize;
        status = cudaFuncSetAttribute(k_dfb_a<true, 6>, a, s6);
        if (status == cudaSuccess) status = cudaFuncSetAttribute(k_dfb_a<false, 6>, a, s6);
        if (status == cudaSuccess) status = cudaFuncSetAttribute(k_dfb_a<true, 8>, a, s8);
        if (status == cudaSuccess) status = cudaFuncSetAttribute(k_dfb_a<false, 8>, a, s8);
    });
    return status;
}

PassParams pass_params(Mode m) {
    switch (m) {
        case FWD: return {1, 0.5f, -0.5f, 1.f, 1.f};       // predict odd, update even
        case INV_ADJ: return {0, 1.f, 1.f, 2.f, -1.f};     // transpose of the inverse stage
        case INV: return {0, 1.f, -1.f, 2.f, 1.f};         // undo update, undo predict
        default: return {1, 0.5f, 0.5f, 1.f, -1.f};        // FWD_ADJ: transpose of the forward stage
    }
}

cudaError_t launch_dfb(const LaunchDfb& L, Mode m, Bases bases, cudaStream_t st, int bthreads) {
    if (L.nblocks == 0) return cudaSuccess;
    const bool syn = (m == INV || m == FWD_ADJ);
    const PassParams pp = pass_params(m);
    if (L.kind == 0) {
        const DfbAJob* j = static_cast<const DfbAJob*>(L.d_jobs);
        if (L.ntaps == 6) {
            if (syn) k_dfb_a<true, 6><<<L.nblocks, 256, AGeo<6>::SMEM, st>>>(j, L.d_block_job, bases, pp);
            else k_dfb_a<false, 6><<<L.nblocks, 256, AGeo<6>::SMEM, st>>>(j, L.d_block_job, bases, pp);
        } else if (L.ntaps == 8) {
            if (syn) k_dfb_a<true, 8><<<L.nblocks, 256, AGeo<8>::SMEM, st>>>(j, L.d_block_job, bases, pp);
            else k_dfb_a<false, 8><<<L.nblocks, 256, AGeo<8>::SMEM, st>>>(j, L.d_block_job, bases, pp);
        } else {
            if (syn) k_dfb_a<true, 4><<<L.nblocks, 256, AGeo<4>::SMEM, st>>>(j, L.d_block_job, bases, pp);
            else k_dfb_a<false, 4><<<L.nblocks, 256, AGeo<4>::SMEM, st>>>(j, L.d_block_job, bases, pp);
        }
    } else {
        const DfbBJob* j = static_cast<const DfbBJob*>(L.d_jobs);
        const bool fo = pp.first_odd != 0;
        // a launch of less than a wave of 128-thread blocks waits on each block's latency:
        // eight warps per tile finish it sooner (unless the caller chose the width)
        const bool wide = bthreads ? bthreads == DFBB_THREADS_WIDE : L.nblocks < 148 * 8;
#define CVC_DFBB_T(S, N, TH)                                                                            \
    do {                                                                                                \
        if (fo) k_dfb_b<S, N, true, TH><<<L.nblocks, TH, 0, st>>>(j, L.d_block_job, bases, pp);          \
        else k_dfb_b<S, N, false, TH><<<L.nblocks, TH, 0, st>>>(j, L.d_block_job, bases, pp);           \
    } while (0)
#define CVC_DFBB(S, N)                                   \
    do {                                                 \
        if (wide) CVC_DFBB_T(S, N, DFBB_THREADS_WIDE);    \
        else CVC_DFBB_T(S, N, DFBB_THREADS);             \
    } while (0)
        if (L.ntaps == 6) {
            if (syn) CVC_DFBB(true, 6);
            else CVC_DFBB(false, 6);
        } else if (L.ntaps == 8) {
            if (syn) CVC_DFBB(true, 8);
            else CVC_DFBB(false, 8);
        } else {
            if (syn) CVC_DFBB(true, 4);
            else CVC_DFBB(false, 4);
        }
#undef CVC_DFBB
#undef CVC_DFBB_T
    }
    return cudaGetLastError();
}

}  // namespace cvc
