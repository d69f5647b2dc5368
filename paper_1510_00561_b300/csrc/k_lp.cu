// k_lp.cu -- Laplacian pyramid level kernels (§2.1, Fig. 1).
//
// One CTA computes a 64 x 64 full-resolution tile of one pyramid level of
// one plane, with periodic extension:
//   analysis:  c = down(x, fa);           d = x - up(c, fs)
//   synthesis: e = c - down(d, fa);       x = d + up(e, fs)
// down(., f) filters separably with f and keeps even samples; up(., f)
// inserts zeros and filters separably with f.  The forward transform and
// its inverse use (fa, fs) = (h, g), the CDF 9/7 analysis / synthesis
// lowpass pair; the adjoints swap the pair ((fa, fs) = (g, h)), because
// down(., f) and up(., f) are transposes of each other for symmetric f.
//
// The tile stages everything through shared memory: the main input with
// its halo (77 x 77), the decimated row pass, the half-resolution tile
// with halo, and the expanded row pass; every input element is read from
// global memory once per tile plus the halo.
//
// The first level of the forward transform and of the inverse runs in single
// precision, centred on a per-tile constant (k_lp_level, CENTRED; see
// lp_level_tile): its numbers are pixels, and centring makes its rounding
// scale with a tile's deviation from its mean.  The other levels accumulate
// in float-float (k_lp_ff:
// error-free TwoSum / FMA-based TwoProd transformations, Dekker 1971 /
// Knuth): the pyramid's DC gain of 2 per level makes coarse levels carry
// numbers up to 2^L * 255, and single-precision roundings of such numbers
// would otherwise reach ~ulp(255) in the detail images and the
// reconstruction.  The taps carry their low-order parts; the analysis forms
// the detail from the unrounded lowpass, and the lowpass images passed
// between synthesis levels are stored as (hi, lo) pairs, so that every
// output rounds once.  The adjoint of the inverse (an analysis with the
// filter pair swapped, whose outputs are gradients) runs in single
// precision (k_lp_level).
#include <mutex>

#include "lp_tile.cuh"

namespace cvc {

// single-precision tile kernel (lp_level_tile): one block per (job, tile)
template <int RA, int RS, bool CENTRED, bool SYN = false>
__global__ void __launch_bounds__(256) k_lp_level(const LpJob* __restrict__ jobs,
                                                  const int* __restrict__ block_job, Bases B) {
    using G = LevelGeo<RA, RS>;
    __shared__ __align__(16) float s_main[G::MN * G::MNS];
    __shared__ __align__(16) float s_a[G::NA];   // row pass (MN x VN), later expanded rows (VN x TS)
    __shared__ float s_v[G::VN * G::VN];
    const LpJob& J = jobs[block_job[blockIdx.x]];
    if (job_idle(B, J.stream)) return;
    lp_level_tile<RA, RS, CENTRED, SYN>(J, blockIdx.x - J.first_block, B, s_main, s_a, s_v);
}

// float-float tile kernel: one block per (job, tile); blocks of streams that take no part return
template <int RA, int RS, bool ANA>
__global__ void __launch_bounds__(256) k_lp_ff(const LpJob* __restrict__ jobs, const int* __restrict__ block_job,
                                               Bases B) {
    extern __shared__ __align__(16) float sm[];
    const LpJob& J = jobs[block_job[blockIdx.x]];
    if (job_idle(B, J.stream)) return;
    lp_ff_tile<RA, RS, ANA>(J, blockIdx.x - J.first_block, B, sm);
}

cudaError_t lp_prepare() {
    // the float-float kernels need more than 48 KB of dynamic shared memory
    static std::once_flag once;
    static cudaError_t status = cudaSuccess;
    std::call_once(once, [] {
        const cudaFuncAttribute a = cudaFuncAttributeMaxDynamicSharedMemorySize;
        status = cudaFuncSetAttribute(k_lp_ff<4, 3, false>, a, (int)ff_smem<4, 3>());
        if (status == cudaSuccess) status = cudaFuncSetAttribute(k_lp_ff<3, 4, false>, a, (int)ff_smem<3, 4>());
        if (status == cudaSuccess) status = cudaFuncSetAttribute(k_lp_ff<4, 3, true>, a, (int)ff_smem<4, 3>());
    });
    return status;
}

cudaError_t launch_lp(const LaunchLp& L, Mode m, Bases bases, cudaStream_t st) {
    if (L.nblocks == 0) return cudaSuccess;
    const bool synth = (m == INV || m == FWD_ADJ);
    const bool swap = (m == FWD_ADJ || m == INV_ADJ);
    dim3 grid(L.nblocks), block(256);
    cudaError_t pe = lp_prepare();
    if (pe != cudaSuccess) return pe;
    // the forward transform and the inverse compute in float-float; the adjoint of the
    // inverse (gradients, checked relative to their own scale) in single precision
    if (!synth && !swap && L.centred)
        k_lp_level<4, 3, true><<<grid, block, 0, st>>>(L.d_jobs, L.d_block_job, bases);
    else if (!synth && !swap) k_lp_ff<4, 3, true><<<grid, block, ff_smem<4, 3>(), st>>>(L.d_jobs, L.d_block_job, bases);
    else if (synth && !swap && L.centred)
        k_lp_level<4, 3, true, true><<<grid, block, 0, st>>>(L.d_jobs, L.d_block_job, bases);
    else if (synth && !swap)
        k_lp_ff<4, 3, false><<<grid, block, ff_smem<4, 3>(), st>>>(L.d_jobs, L.d_block_job, bases);
    else if (!synth && swap) k_lp_level<3, 4, false><<<grid, block, 0, st>>>(L.d_jobs, L.d_block_job, bases);
    else k_lp_ff<3, 4, false><<<grid, block, ff_smem<3, 4>(), st>>>(L.d_jobs, L.d_block_job, bases);
    return cudaGetLastError();
}

}  // namespace cvc
