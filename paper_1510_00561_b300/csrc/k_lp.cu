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
// The forward transform and the inverse accumulate in float-float (k_lp_ff:
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

// single-precision analysis tile: cout = down(main, fa); out = main - up(cout, fs)
template <int RA, int RS>
__global__ void __launch_bounds__(256) k_lp_level(const LpJob* __restrict__ jobs,
                                                  const int* __restrict__ block_job, Bases B) {
    constexpr int T = LP_TILE;
    constexpr int MLO = -(RS / 2);
    constexpr int MHI = (T - 1 + RS) / 2;
    constexpr int VN = MHI - MLO + 1;
    constexpr int MN = 2 * (VN - 1) + 2 * RA + 1;
    constexpr int Y0 = 2 * MLO - RA;  // main tile origin relative to the output tile origin
    constexpr int NA = (MN * VN > VN * T) ? MN * VN : VN * T;
    constexpr int MNS = MN + (MN & 1);   // even row stride: the row pass reads its windows in pairs

    __shared__ __align__(16) float s_main[MN * MNS];
    __shared__ __align__(16) float s_a[NA];   // row pass (MN x VN), later expanded rows (VN x T)
    __shared__ float s_v[VN * VN];

    const int jid = block_job[blockIdx.x];
    const LpJob& J = jobs[jid];
    if (job_idle(B, J.stream)) return;
    const int tile = blockIdx.x - J.first_block;
    const int ty = tile / J.tiles_x, tx = tile - ty * J.tiles_x;
    const int y0 = ty * T, x0 = tx * T;
    const int m0 = y0 / 2, n0 = x0 / 2;
    const int H = J.H, W = J.W, Hh = H / 2, Wh = W / 2;
    const float* mainp = base_ptr(B, J.main.b) + J.main.off;
    const int mrs = J.main.rs;

    lp_stage<MN, MNS>(s_main, mainp, mrs, y0 + Y0, x0 + Y0, H, W);
    lp_cp_async_wait_all();
    __syncthreads();
    // decimating row pass: s_a[r][n'] = sum_b fa[b] main[r][2n' + RA - b]; the window
    // main[r][2n' + j], j = 0 .. 2 RA, starts at an even offset: RA pairs and one more
    for (int i = threadIdx.x; i < MN * VN; i += blockDim.x) {
        int r = i / VN, n = i - r * VN;
        const float* w = s_main + r * MNS + 2 * n;
        float x[2 * RA + 1];
#pragma unroll
        for (int j = 0; j < RA; j++) {
            const float2 pr = *reinterpret_cast<const float2*>(w + 2 * j);
            x[2 * j] = pr.x;
            x[2 * j + 1] = pr.y;
        }
        x[2 * RA] = w[2 * RA];
        float acc = 0.f;
#pragma unroll
        for (int b = -RA; b <= RA; b++) acc = fmaf(tap_a<RA>(b), x[RA - b], acc);
        s_a[i] = acc;
    }
    __syncthreads();
    // decimating column pass -> half-resolution values v on [m0+MLO, m0+MHI] x [n0+MLO, n0+MHI]
    for (int i = threadIdx.x; i < VN * VN; i += blockDim.x) {
        int m = i / VN, n = i - m * VN;
        float acc = 0.f;
#pragma unroll
        for (int a = -RA; a <= RA; a++) acc = fmaf(tap_a<RA>(a), s_a[(2 * m + RA - a) * VN + n], acc);
        s_v[i] = acc;
    }
    __syncthreads();
    {
        // interior 32 x 32 of v is this tile's share of the lowpass output
        float* coutp = base_ptr(B, J.cout.b) + J.cout.off;
        for (int i = threadIdx.x; i < (T / 2) * (T / 2); i += blockDim.x) {
            int m = i / (T / 2), n = i - m * (T / 2);
            int gm = m0 + m, gn = n0 + n;
            if (gm < Hh && gn < Wh) coutp[(long long)gm * J.cout.rs + gn] = s_v[(m - MLO) * VN + (n - MLO)];
        }
    }
    // expanding row pass, by output pairs (x = 2p, 2p + 1):
    //   s_a[m][x] = sum_{t : x - t even} fs[t] v[m][(x - t)/2 - MLO]
    for (int i = threadIdx.x; i < VN * (T / 2); i += blockDim.x) {
        const int m = i / (T / 2), p = i - m * (T / 2);
        const float* vr = s_v + m * VN + p - MLO;
        float ev = 0.f, od = 0.f;
#pragma unroll
        for (int t = -RS; t <= RS; t++) {
            if ((t & 1) == 0) ev = fmaf(tap_s<RS>(t), vr[-(t / 2)], ev);               // x = 2p
            else od = fmaf(tap_s<RS>(t), vr[(1 - t) / 2], od);                           // x = 2p + 1
        }
        *reinterpret_cast<float2*>(s_a + m * T + 2 * p) = make_float2(ev, od);
    }
    __syncthreads();
    // expanding column pass by output pairs (y = 2p, 2p + 1) and the combination with the main input
    float* outp = base_ptr(B, J.out.b) + J.out.off;
    for (int i = threadIdx.x; i < (T / 2) * T; i += blockDim.x) {
        const int p = i / T, x = i - p * T;
        const float* ar = s_a + (p - MLO) * T + x;
        float ev = 0.f, od = 0.f;
#pragma unroll
        for (int t = -RS; t <= RS; t++) {
            if ((t & 1) == 0) ev = fmaf(tap_s<RS>(t), ar[-(t / 2) * T], ev);
            else od = fmaf(tap_s<RS>(t), ar[((1 - t) / 2) * T], od);
        }
        const int gx = x0 + x;
#pragma unroll
        for (int h = 0; h < 2; h++) {
            const int y = 2 * p + h, gy = y0 + y;
            if (gy < H && gx < W) {
                const float acc = h ? od : ev;
                const float mv = s_main[(y - Y0) * MNS + (x - Y0)];
                outp[(long long)gy * J.out.rs + gx] = mv - acc;
            }
        }
    }
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
    if (!synth && !swap) k_lp_ff<4, 3, true><<<grid, block, ff_smem<4, 3>(), st>>>(L.d_jobs, L.d_block_job, bases);
    else if (synth && !swap)
        k_lp_ff<4, 3, false><<<grid, block, ff_smem<4, 3>(), st>>>(L.d_jobs, L.d_block_job, bases);
    else if (!synth && swap) k_lp_level<3, 4><<<grid, block, 0, st>>>(L.d_jobs, L.d_block_job, bases);
    else k_lp_ff<3, 4, false><<<grid, block, ff_smem<3, 4>(), st>>>(L.d_jobs, L.d_block_job, bases);
    return cudaGetLastError();
}

}  // namespace cvc
