// k_lp.cu -- Laplacian pyramid level kernels (§2.1, Fig. 1).
//
// One CTA computes a 64 x 64 full-resolution tile of one pyramid level of
// one plane, with periodic extension.  Two kernels share one body:
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
// Synthesis accumulates in float-float (error-free TwoSum / FMA-based
// TwoProd transformations, Dekker 1971 / Knuth): the pyramid's DC gain of 2
// per level makes coarse levels carry numbers up to 2^L * 255, and each
// level's single-precision roundings would otherwise add ~ulp(255) to the
// reconstruction; with compensated sums only the stored values round.
#include <mutex>

#include "cvc_internal.cuh"

namespace cvc {

// CDF 9/7 lowpass pair normalised to DC gain sqrt(2) (published values,
// 12 significant digits): analysis h (taps -4..4), synthesis g (-3..3).
__constant__ float c_h[9] = {0.037828455507f, -0.023849465020f, -0.110624404418f, 0.377402855613f,
                             0.852698679009f,  0.377402855613f, -0.110624404418f, -0.023849465020f,
                             0.037828455507f};
__constant__ float c_g[7] = {-0.064538882629f, -0.040689417609f, 0.418092273222f, 0.788485616406f,
                             0.418092273222f,  -0.040689417609f, -0.064538882629f};

__device__ __forceinline__ int wrap_idx(int a, int n) {
    if ((unsigned)a < (unsigned)n) return a;
    int r = a % n;
    return r < 0 ? r + n : r;
}

// 4-byte asynchronous global -> shared copies (all of a tile's staging in flight at once)
__device__ __forceinline__ void lp_cp_async4(float* dst, const float* src) {
    const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(d), "l"(src) : "memory");
}
__device__ __forceinline__ void lp_cp_async_wait_all() {
    asm volatile("cp.async.commit_group;\ncp.async.wait_group 0;\n" ::: "memory");
}

// stage the MN x MN main tile at (ty0, tx0) (periodic) with row stride MNS: a warp per
// row, lanes along it; a tile whose columns do not wrap takes no per-element index arithmetic
template <int MN, int MNS = MN>
__device__ __forceinline__ void lp_stage(float* s_main, const float* mainp, int mrs, int ty0, int tx0, int H, int W) {
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nwarp = blockDim.x >> 5;
    const bool inner = tx0 >= 0 && tx0 + MN <= W;
    for (int r = warp; r < MN; r += nwarp) {
        const float* row = mainp + (long long)wrap_idx(ty0 + r, H) * mrs;
        float* dst = s_main + r * MNS;
        if (inner) {
            const float* src = row + tx0;
            for (int c = lane; c < MN; c += 32) lp_cp_async4(dst + c, src + c);
        } else {
            for (int c = lane; c < MN; c += 32) lp_cp_async4(dst + c, row + wrap_idx(tx0 + c, W));
        }
    }
}

template <int RA>
__device__ __forceinline__ float tap_a(int t) { return RA == 4 ? c_h[t + 4] : c_g[t + 3]; }
template <int RS>
__device__ __forceinline__ float tap_s(int t) { return RS == 3 ? c_g[t + 3] : c_h[t + 4]; }

template <int RA, int RS, bool SYNTH>
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
    const float* cinp = SYNTH ? base_ptr(B, J.cin.b) + J.cin.off : nullptr;
    for (int i = threadIdx.x; i < VN * VN; i += blockDim.x) {
        int m = i / VN, n = i - m * VN;
        float acc = 0.f;
#pragma unroll
        for (int a = -RA; a <= RA; a++) acc = fmaf(tap_a<RA>(a), s_a[(2 * m + RA - a) * VN + n], acc);
        if (SYNTH) {
            int gm = wrap_idx(m0 + MLO + m, Hh), gn = wrap_idx(n0 + MLO + n, Wh);
            acc = cinp[(long long)gm * J.cin.rs + gn] - acc;
        }
        s_v[i] = acc;
    }
    __syncthreads();
    if (!SYNTH) {
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
                outp[(long long)gy * J.out.rs + gx] = SYNTH ? mv + acc : mv - acc;
            }
        }
    }
}

// ------------------------------------------------- float-float helpers
// (hi, lo) accumulators; __fadd_rn / __fmul_rn keep the compiler from
// contracting the error-free transformations into FMAs.
__device__ __forceinline__ void ff_add(float& hi, float& lo, float x) {
    float s = __fadd_rn(hi, x);
    float bb = __fsub_rn(s, hi);
    float e = __fadd_rn(__fsub_rn(hi, __fsub_rn(s, bb)), __fsub_rn(x, bb));
    hi = s;
    lo = __fadd_rn(lo, e);
}
// (hi, lo) += f * (xh + xl)
__device__ __forceinline__ void ff_fma(float& hi, float& lo, float f, float xh, float xl) {
    float p = __fmul_rn(f, xh);
    float pe = fmaf(f, xh, -p);
    ff_add(hi, lo, p);
    lo = fmaf(f, xl, __fadd_rn(lo, pe));
}
__device__ __forceinline__ void ff_norm(float& hi, float& lo) {
    float s = __fadd_rn(hi, lo);
    lo = __fsub_rn(lo, __fsub_rn(s, hi));
    hi = s;
}

// The same transformations on two independent lanes at once (paired FP32
// instructions; each lane rounds exactly as the scalar sequence above).
__device__ __forceinline__ float2 neg2(float2 a) { return make_float2(-a.x, -a.y); }
__device__ __forceinline__ void ff2_add(float2& hi, float2& lo, float2 x) {
    const float2 s = __fadd2_rn(hi, x);
    const float2 bb = __fadd2_rn(s, neg2(hi));
    const float2 e = __fadd2_rn(__fadd2_rn(hi, neg2(__fadd2_rn(s, neg2(bb)))), __fadd2_rn(x, neg2(bb)));
    hi = s;
    lo = __fadd2_rn(lo, e);
}
__device__ __forceinline__ void ff2_fma(float2& hi, float2& lo, float f, float2 xh, float2 xl) {
    const float2 ff = make_float2(f, f);
    const float2 p = __fmul2_rn(ff, xh);
    const float2 pe = __ffma2_rn(ff, xh, neg2(p));
    ff2_add(hi, lo, p);
    lo = __ffma2_rn(ff, xl, __fadd2_rn(lo, pe));
}

// Synthesis tile with float-float intermediates (dynamic shared memory):
//   e = cin - down(main, fa);  out = main + up(e, fs)
template <int RA, int RS>
__global__ void __launch_bounds__(256) k_lp_synth_ff(const LpJob* __restrict__ jobs,
                                                     const int* __restrict__ block_job, Bases B) {
    constexpr int T = LP_TILE;
    constexpr int MLO = -(RS / 2);
    constexpr int MHI = (T - 1 + RS) / 2;
    constexpr int VN = MHI - MLO + 1;
    constexpr int MN = 2 * (VN - 1) + 2 * RA + 1;
    constexpr int Y0 = 2 * MLO - RA;
    constexpr int NA = (MN * VN > VN * T) ? MN * VN : VN * T;
    // the main tile's rows have an even stride and the float-float arrays start on
    // 16-byte boundaries, so that the passes below move pairs and quadruples
    constexpr int MNS = MN + (MN & 1), OA = (MN * MNS + 3) & ~3, NA4 = (NA + 3) & ~3;
    extern __shared__ __align__(16) float sm[];
    float* s_main = sm;                 // MN rows of MNS
    float* s_ah = s_main + OA;          // NA
    float* s_al = s_ah + NA4;           // NA
    float* s_vh = s_al + NA4;           // VN * VN
    float* s_vl = s_vh + VN * VN;       // VN * VN

    const int jid = block_job[blockIdx.x];
    const LpJob& J = jobs[jid];
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
    // Every pass computes two outputs per thread with paired instructions.
    // decimating row pass, row pairs (ra, rb) (an odd last row pairs with itself), so that
    // consecutive threads read consecutive columns as in a scalar pass
    constexpr int NR = (MN + 1) / 2, NM = (VN + 1) / 2;
    const float2 zero2 = make_float2(0.f, 0.f);
    for (int i = threadIdx.x; i < NR * VN; i += blockDim.x) {
        const int q = i / VN, n = i - q * VN;
        const int ra = 2 * q, rb = min(2 * q + 1, MN - 1);
        // the window x[2n + j], j = 0 .. 2 RA, of both rows (even offsets: RA pairs and one more)
        const float* wa = s_main + ra * MNS + 2 * n;
        const float* wb = s_main + rb * MNS + 2 * n;
        float va[2 * RA + 1], vb[2 * RA + 1];
#pragma unroll
        for (int j = 0; j < RA; j++) {
            const float2 pa = *reinterpret_cast<const float2*>(wa + 2 * j);
            const float2 pb = *reinterpret_cast<const float2*>(wb + 2 * j);
            va[2 * j] = pa.x; va[2 * j + 1] = pa.y;
            vb[2 * j] = pb.x; vb[2 * j + 1] = pb.y;
        }
        va[2 * RA] = wa[2 * RA];
        vb[2 * RA] = wb[2 * RA];
        float2 hi = zero2, lo = zero2;
#pragma unroll
        for (int b = -RA; b <= RA; b++) ff2_fma(hi, lo, tap_a<RA>(b), make_float2(va[RA - b], vb[RA - b]), zero2);
        s_ah[ra * VN + n] = hi.x;
        s_al[ra * VN + n] = lo.x;
        if (rb != ra) {
            s_ah[rb * VN + n] = hi.y;
            s_al[rb * VN + n] = lo.y;
        }
    }
    __syncthreads();
    // decimating column pass over row pairs (ma, mb), then e = cin - down(main) (normalised float-float)
    const float* cinp = base_ptr(B, J.cin.b) + J.cin.off;
    for (int i = threadIdx.x; i < NM * VN; i += blockDim.x) {
        const int q = i / VN, n = i - q * VN;
        const int ma = 2 * q, mb = min(2 * q + 1, VN - 1);
        float2 hi = zero2, lo = zero2;
#pragma unroll
        for (int a = -RA; a <= RA; a++) {
            const int ka = (2 * ma + RA - a) * VN + n, kb = (2 * mb + RA - a) * VN + n;
            ff2_fma(hi, lo, tap_a<RA>(a), make_float2(s_ah[ka], s_ah[kb]), make_float2(s_al[ka], s_al[kb]));
        }
        const int gn = wrap_idx(n0 + MLO + n, Wh);
        float2 eh = make_float2(cinp[(long long)wrap_idx(m0 + MLO + ma, Hh) * J.cin.rs + gn],
                                cinp[(long long)wrap_idx(m0 + MLO + mb, Hh) * J.cin.rs + gn]);
        float2 el = zero2;
        ff2_add(eh, el, neg2(hi));
        el = __fadd2_rn(el, neg2(lo));
        const float2 sn = __fadd2_rn(eh, el);
        el = __fadd2_rn(el, neg2(__fadd2_rn(sn, neg2(eh))));
        eh = sn;
        s_vh[ma * VN + n] = eh.x;
        s_vl[ma * VN + n] = el.x;
        if (mb != ma) {
            s_vh[mb * VN + n] = eh.y;
            s_vl[mb * VN + n] = el.y;
        }
    }
    __syncthreads();
    // expanding row pass: output pairs x = 2p, 2p + 1 for p = 2w and 2w + 1
    for (int i = threadIdx.x; i < VN * (T / 4); i += blockDim.x) {
        const int m = i / (T / 4), w = i - m * (T / 4);
        const int kb = m * VN + 2 * w - MLO;
        float2 eh = zero2, el = zero2, oh = zero2, ol = zero2;
#pragma unroll
        for (int t = -RS; t <= RS; t++) {
            if ((t & 1) == 0) {
                const int k = kb - t / 2;
                ff2_fma(eh, el, tap_s<RS>(t), make_float2(s_vh[k], s_vh[k + 1]), make_float2(s_vl[k], s_vl[k + 1]));
            } else {
                const int k = kb + (1 - t) / 2;
                ff2_fma(oh, ol, tap_s<RS>(t), make_float2(s_vh[k], s_vh[k + 1]), make_float2(s_vl[k], s_vl[k + 1]));
            }
        }
        *reinterpret_cast<float4*>(s_ah + m * T + 4 * w) = make_float4(eh.x, oh.x, eh.y, oh.y);
        *reinterpret_cast<float4*>(s_al + m * T + 4 * w) = make_float4(el.x, ol.x, el.y, ol.y);
    }
    __syncthreads();
    // expanding column pass: output rows 2p, 2p + 1 for the column pair (2w, 2w + 1), plus the main input
    float* outp = base_ptr(B, J.out.b) + J.out.off;
    for (int i = threadIdx.x; i < (T / 2) * (T / 2); i += blockDim.x) {
        const int p = i / (T / 2), w = i - p * (T / 2);
        const int x = 2 * w;
        const int kb = (p - MLO) * T + x;
        float2 eh = zero2, el = zero2, oh = zero2, ol = zero2;
#pragma unroll
        for (int t = -RS; t <= RS; t++) {
            if ((t & 1) == 0) {
                const int k = kb - (t / 2) * T;
                ff2_fma(eh, el, tap_s<RS>(t), *reinterpret_cast<const float2*>(s_ah + k),
                        *reinterpret_cast<const float2*>(s_al + k));
            } else {
                const int k = kb + ((1 - t) / 2) * T;
                ff2_fma(oh, ol, tap_s<RS>(t), *reinterpret_cast<const float2*>(s_ah + k),
                        *reinterpret_cast<const float2*>(s_al + k));
            }
        }
        const int gx = x0 + x;
#pragma unroll
        for (int h = 0; h < 2; h++) {
            const int y = 2 * p + h, gy = y0 + y;
            if (gy >= H) continue;
            float2 hi = h ? oh : eh, lo = h ? ol : el;
            const float* mrow = s_main + (y - Y0) * MNS + (x - Y0);
            ff2_add(hi, lo, make_float2(mrow[0], mrow[1]));
            const float2 o = __fadd2_rn(hi, lo);
            float* orow = outp + (long long)gy * J.out.rs;
            if (gx < W) orow[gx] = o.x;
            if (gx + 1 < W) orow[gx + 1] = o.y;
        }
    }
}

template <int RA, int RS>
constexpr size_t synth_ff_smem() {
    constexpr int T = LP_TILE;
    constexpr int MLO = -(RS / 2);
    constexpr int MHI = (T - 1 + RS) / 2;
    constexpr int VN = MHI - MLO + 1;
    constexpr int MN = 2 * (VN - 1) + 2 * RA + 1;
    constexpr int NA = (MN * VN > VN * T) ? MN * VN : VN * T;
    constexpr int MNS = MN + (MN & 1), OA = (MN * MNS + 3) & ~3, NA4 = (NA + 3) & ~3;
    return sizeof(float) * (size_t)(OA + 2 * NA4 + 2 * VN * VN);
}

cudaError_t lp_prepare() {
    // the float-float synthesis kernels need more than 48 KB of dynamic shared memory
    static std::once_flag once;
    static cudaError_t status = cudaSuccess;
    std::call_once(once, [] {
        status = cudaFuncSetAttribute(k_lp_synth_ff<4, 3>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      (int)synth_ff_smem<4, 3>());
        if (status == cudaSuccess)
            status = cudaFuncSetAttribute(k_lp_synth_ff<3, 4>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                          (int)synth_ff_smem<3, 4>());
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
    if (!synth && !swap) k_lp_level<4, 3, false><<<grid, block, 0, st>>>(L.d_jobs, L.d_block_job, bases);
    else if (synth && !swap)
        k_lp_synth_ff<4, 3><<<grid, block, synth_ff_smem<4, 3>(), st>>>(L.d_jobs, L.d_block_job, bases);
    else if (!synth && swap) k_lp_level<3, 4, false><<<grid, block, 0, st>>>(L.d_jobs, L.d_block_job, bases);
    else k_lp_synth_ff<3, 4><<<grid, block, synth_ff_smem<3, 4>(), st>>>(L.d_jobs, L.d_block_job, bases);
    return cudaGetLastError();
}

}  // namespace cvc
