// lp_tile.cuh -- the Laplacian-pyramid tile (§2.1, Fig. 1) as a device
// function, shared by the per-level kernels (k_lp.cu) and the tail kernel
// that runs a plane's coarse levels in one block (k_tail.cu).
//
// One tile is a 64 x 64 full-resolution output block of one pyramid level of
// one plane, with periodic extension:
//   analysis:  c = down(x, fa);           d = x - up(c, fs)
//   synthesis: e = c - down(d, fa);       x = d + up(e, fs)
// staged through shared memory (see k_lp.cu).  A tile's input may live in
// global memory (asynchronous copies) or, inside the tail kernel, in shared
// memory (plain copies); every output element is computed by the same
// sequence of operations either way, so both give the same bits.
#pragma once
#include "cvc_internal.cuh"

namespace cvc {


// CDF 9/7 lowpass pair normalised to DC gain sqrt(2) (published values,
// 12 significant digits): analysis h (taps -4..4), synthesis g (-3..3).
// Each tap is held as a float and, for the float-float synthesis, the float
// nearest its remainder: the remainder matters there because a level-j
// lowpass carries numbers up to 2^j * 255, and the taps' single-precision
// representation error (up to 2^-25 relative) times such numbers is
// ~ulp(255) at the coarse levels.
#define CVC_H4 0.037828455507
#define CVC_H3 -0.023849465020
#define CVC_H2 -0.110624404418
#define CVC_H1 0.377402855613
#define CVC_H0 0.852698679009
#define CVC_G3 -0.064538882629
#define CVC_G2 -0.040689417609
#define CVC_G1 0.418092273222
#define CVC_G0 0.788485616406
#define CVC_LO(t) ((float)((t) - (double)(float)(t)))
static __constant__ float c_h[9] = {(float)CVC_H4, (float)CVC_H3, (float)CVC_H2, (float)CVC_H1, (float)CVC_H0,
                             (float)CVC_H1, (float)CVC_H2, (float)CVC_H3, (float)CVC_H4};
static __constant__ float c_g[7] = {(float)CVC_G3, (float)CVC_G2, (float)CVC_G1, (float)CVC_G0,
                             (float)CVC_G1, (float)CVC_G2, (float)CVC_G3};
static __constant__ float c_hl[9] = {CVC_LO(CVC_H4), CVC_LO(CVC_H3), CVC_LO(CVC_H2), CVC_LO(CVC_H1), CVC_LO(CVC_H0),
                              CVC_LO(CVC_H1), CVC_LO(CVC_H2), CVC_LO(CVC_H3), CVC_LO(CVC_H4)};
static __constant__ float c_gl[7] = {CVC_LO(CVC_G3), CVC_LO(CVC_G2), CVC_LO(CVC_G1), CVC_LO(CVC_G0),
                              CVC_LO(CVC_G1), CVC_LO(CVC_G2), CVC_LO(CVC_G3)};

__device__ __forceinline__ int wrap_idx(int a, int n) {
    if ((unsigned)a < (unsigned)n) return a;
    const int b = a < 0 ? a + n : a - n;   // one period outside: no division
    if ((unsigned)b < (unsigned)n) return b;
    const int r = a % n;
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
    const bool from_shared = __isShared(mainp);   // a tail kernel's resident image: plain copies
    for (int r = warp; r < MN; r += nwarp) {
        const float* row = mainp + (long long)wrap_idx(ty0 + r, H) * mrs;
        float* dst = s_main + r * MNS;
        if (from_shared) {
            for (int c = lane; c < MN; c += 32) dst[c] = row[wrap_idx(tx0 + c, W)];
        } else if (inner) {
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
// the taps' low-order parts
template <int RA>
__device__ __forceinline__ float tapl_a(int t) { return RA == 4 ? c_hl[t + 4] : c_gl[t + 3]; }
template <int RS>
__device__ __forceinline__ float tapl_s(int t) { return RS == 3 ? c_gl[t + 3] : c_hl[t + 4]; }

// ------------------------------------------------- float-float helpers
// (hi, lo) accumulators on two independent lanes at once (paired FP32
// instructions); __fadd2_rn / __fmul2_rn keep the compiler from contracting
// the error-free transformations into FMAs.
__device__ __forceinline__ float2 neg2(float2 a) { return make_float2(-a.x, -a.y); }
__device__ __forceinline__ void ff2_add(float2& hi, float2& lo, float2 x) {
    const float2 s = __fadd2_rn(hi, x);
    const float2 bb = __fadd2_rn(s, neg2(hi));
    const float2 e = __fadd2_rn(__fadd2_rn(hi, neg2(__fadd2_rn(s, neg2(bb)))), __fadd2_rn(x, neg2(bb)));
    hi = s;
    lo = __fadd2_rn(lo, e);
}
// ------------------------------------------------- fixed-grid compensated sums
// A pass accumulates sum_k f_k x_k as a pair (sh, sl): every product is rounded
// to a multiple of a grid step G (a power of two) by one fused multiply-add with
// the constant C = 1.5 * 2^23 * G, whose unit in the last place is G, and the
// rest of the product goes to sl.  Sums of multiples of G below 2^24 G are
// exact, so sh carries no rounding at all and sl only small terms (|sl| below a
// few G, a few dozen roundings of 2^-24 |sl| each): the pair holds the sum to
// about 2^-37 of the bound that chose G, at 7 paired instructions per tap where
// a float-float (TwoProduct + TwoSum) update takes 11.
// grid_c(B): C for G = 2^(ceil(log2 B) - 21), B >= every product and partial sum.
__device__ __forceinline__ float2 grid_c(float bound) {
    const int e = (__float_as_int(bound) >> 23) & 255;   // biased exponent of |bound|
    const int ec = min(e + 3, 254);                      // C = 1.5 * 2^(e - 124)
    const float c = __int_as_float((ec << 23) | 0x400000);
    return make_float2(c, c);
}
// (sh, sl) += (f + fl) * (xh + xl), dropping only fl * xl
__device__ __forceinline__ void gacc(float2& sh, float2& sl, float2 c, float f, float fl, float2 xh, float2 xl) {
    const float2 ff = make_float2(f, f);
    const float2 ph = __fadd2_rn(__ffma2_rn(ff, xh, c), neg2(c));   // f xh on the grid
    const float2 pl = __ffma2_rn(ff, xh, neg2(ph));                 // the rest of f xh
    sh = __fadd2_rn(sh, ph);
    sl = __fadd2_rn(sl, pl);
    sl = __ffma2_rn(ff, xl, sl);
    sl = __ffma2_rn(make_float2(fl, fl), xh, sl);
}
// the same with a single-precision x
__device__ __forceinline__ void gacc1(float2& sh, float2& sl, float2 c, float f, float fl, float2 x) {
    const float2 ff = make_float2(f, f);
    const float2 ph = __fadd2_rn(__ffma2_rn(ff, x, c), neg2(c));
    const float2 pl = __ffma2_rn(ff, x, neg2(ph));
    sh = __fadd2_rn(sh, ph);
    sl = __fadd2_rn(sl, pl);
    sl = __ffma2_rn(make_float2(fl, fl), x, sl);
}
// (hi, lo) <- TwoSum(hi, lo): hi the rounded sum, lo its exact error (any magnitudes)
__device__ __forceinline__ void two_sum2(float2& hi, float2& lo) {
    const float2 s = __fadd2_rn(hi, lo);
    const float2 bb = __fadd2_rn(s, neg2(hi));
    lo = __fadd2_rn(__fadd2_rn(hi, neg2(__fadd2_rn(s, neg2(bb)))), __fadd2_rn(lo, neg2(bb)));
    hi = s;
}
__device__ __forceinline__ float lp_warp_max(float v) {
#pragma unroll
    for (int o = 16; o; o >>= 1) v = fmaxf(v, __shfl_xor_sync(0xffffffffu, v, o));
    return v;
}

// One tile with compensated intermediates (sm: ff_smem<RA, RS>() bytes of shared memory):
//   synthesis (ANA = false): e = cin - down(main, fa);  out = main + up(e, fs)
//   analysis  (ANA = true):  e = -down(main, fa), cout = -e (rounded);  out = main + up(e, fs)
// so that the detail image of the analysis carries only its own rounding:
// the lowpass it is computed from is not rounded first.  The two decimating
// passes sum on a grid chosen from the largest magnitude of the staged tile,
// the two expanding passes on one chosen from the largest |e| (a block-wide
// maximum each); e itself and the output take float-float additions.
template <int RA, int RS, bool ANA>
__device__ __forceinline__ void lp_ff_tile(const LpJob& J, int tile, const Bases& B, float* sm) {
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
    float* s_main = sm;                 // MN rows of MNS
    float* s_ah = s_main + OA;          // NA
    float* s_al = s_ah + NA4;           // NA
    float* s_vh = s_al + NA4;           // VN * VN
    float* s_vl = s_vh + VN * VN;       // VN * VN
    float* s_red = s_vl + VN * VN;      // 16: per-warp maxima of the two grids

    const int ty = tile / J.tiles_x, tx = tile - ty * J.tiles_x;
    const int y0 = ty * T, x0 = tx * T;
    const int m0 = y0 / 2, n0 = x0 / 2;
    const int H = J.H, W = J.W, Hh = H / 2, Wh = W / 2;
    const float* mainp = base_ptr(B, J.main.b) + J.main.off;
    const int mrs = J.main.rs;
    lp_stage<MN, MNS>(s_main, mainp, mrs, y0 + Y0, x0 + Y0, H, W);
    lp_cp_async_wait_all();
    __syncthreads();
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nwarp = blockDim.x >> 5;
    // the grid of the decimating passes: products and partial sums stay below
    // sum|h| max|a| <= 1.96^2 max|main| < 4 max|main|
    float2 c1;
    {
        float m = 0.f;
        for (int r = warp; r < MN; r += nwarp)
            for (int c = lane; c < MN; c += 32) m = fmaxf(m, fabsf(s_main[r * MNS + c]));
        m = lp_warp_max(m);
        if (lane == 0) s_red[warp] = m;
        __syncthreads();
        for (int w = 0; w < nwarp; w++) m = fmaxf(m, s_red[w]);
        c1 = grid_c(4.f * m);
    }
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
        for (int b = -RA; b <= RA; b++) gacc1(hi, lo, c1, tap_a<RA>(b), tapl_a<RA>(b), make_float2(va[RA - b], vb[RA - b]));
        s_ah[ra * VN + n] = hi.x;
        s_al[ra * VN + n] = lo.x;
        if (rb != ra) {
            s_ah[rb * VN + n] = hi.y;
            s_al[rb * VN + n] = lo.y;
        }
    }
    __syncthreads();
    // decimating column pass over row pairs (ma, mb), then e = cin - down(main) (normalised float-float);
    // the analysis takes e = -down(main) and writes the interior of down(main) as its lowpass output
    const float* cinp = ANA ? nullptr : base_ptr(B, J.cin.b) + J.cin.off;
    const float* cinlp = !ANA && J.cin_lo.b >= 0 ? base_ptr(B, J.cin_lo.b) + J.cin_lo.off : nullptr;
    float* coutp = ANA ? base_ptr(B, J.cout.b) + J.cout.off : nullptr;
    float me = 0.f;   // this thread's largest |e|
    for (int i = threadIdx.x; i < NM * VN; i += blockDim.x) {
        const int q = i / VN, n = i - q * VN;
        const int ma = 2 * q, mb = min(2 * q + 1, VN - 1);
        float2 hi = zero2, lo = zero2;
#pragma unroll
        for (int a = -RA; a <= RA; a++) {
            const int ka = (2 * ma + RA - a) * VN + n, kb = (2 * mb + RA - a) * VN + n;
            gacc(hi, lo, c1, tap_a<RA>(a), tapl_a<RA>(a), make_float2(s_ah[ka], s_ah[kb]), make_float2(s_al[ka], s_al[kb]));
        }
        float2 eh, el;
        if (ANA) {
            eh = neg2(hi);
            el = neg2(lo);
        } else {
            const int gn = wrap_idx(n0 + MLO + n, Wh);
            const int gma = wrap_idx(m0 + MLO + ma, Hh), gmb = wrap_idx(m0 + MLO + mb, Hh);
            eh = make_float2(cinp[(long long)gma * J.cin.rs + gn], cinp[(long long)gmb * J.cin.rs + gn]);
            el = zero2;
            if (cinlp)
                el = make_float2(cinlp[(long long)gma * J.cin_lo.rs + gn], cinlp[(long long)gmb * J.cin_lo.rs + gn]);
            ff2_add(eh, el, neg2(hi));
            el = __fadd2_rn(el, neg2(lo));
        }
        two_sum2(eh, el);
        me = fmaxf(me, fmaxf(fabsf(eh.x), fabsf(eh.y)));
        if (ANA) {
            // this tile's share of the lowpass: half-resolution rows / columns [m0, m0 + T/2) x [n0, n0 + T/2)
            const int gn = n0 + MLO + n;
            if (n >= -MLO && n < -MLO + T / 2 && gn < Wh) {
                const int ga = m0 + MLO + ma, gb = m0 + MLO + mb;
                if (ma >= -MLO && ma < -MLO + T / 2 && ga < Hh) coutp[(long long)ga * J.cout.rs + gn] = -eh.x;
                if (mb != ma && mb >= -MLO && mb < -MLO + T / 2 && gb < Hh) coutp[(long long)gb * J.cout.rs + gn] = -eh.y;
            }
        }
        s_vh[ma * VN + n] = eh.x;
        s_vl[ma * VN + n] = el.x;
        if (mb != ma) {
            s_vh[mb * VN + n] = eh.y;
            s_vl[mb * VN + n] = el.y;
        }
    }
    me = lp_warp_max(me);
    if (lane == 0) s_red[8 + warp] = me;
    __syncthreads();
    // the grid of the expanding passes: each output phase has sum|g| < 1, so products
    // and partial sums of both passes stay below max|e| (plus the low parts)
    float2 c2;
    {
        float m = 0.f;
        for (int w = 0; w < nwarp; w++) m = fmaxf(m, s_red[8 + w]);
        c2 = grid_c(2.f * m);
    }
    // expanding row pass: output pairs x = 2p, 2p + 1 for p = 2w and 2w + 1
    for (int i = threadIdx.x; i < VN * (T / 4); i += blockDim.x) {
        const int m = i / (T / 4), w = i - m * (T / 4);
        const int kb = m * VN + 2 * w - MLO;
        float2 eh = zero2, el = zero2, oh = zero2, ol = zero2;
#pragma unroll
        for (int t = -RS; t <= RS; t++) {
            if ((t & 1) == 0) {
                const int k = kb - t / 2;
                gacc(eh, el, c2, tap_s<RS>(t), tapl_s<RS>(t), make_float2(s_vh[k], s_vh[k + 1]),
                     make_float2(s_vl[k], s_vl[k + 1]));
            } else {
                const int k = kb + (1 - t) / 2;
                gacc(oh, ol, c2, tap_s<RS>(t), tapl_s<RS>(t), make_float2(s_vh[k], s_vh[k + 1]),
                     make_float2(s_vl[k], s_vl[k + 1]));
            }
        }
        *reinterpret_cast<float4*>(s_ah + m * T + 4 * w) = make_float4(eh.x, oh.x, eh.y, oh.y);
        *reinterpret_cast<float4*>(s_al + m * T + 4 * w) = make_float4(el.x, ol.x, el.y, ol.y);
    }
    __syncthreads();
    // expanding column pass: output rows 2p, 2p + 1 for the column pair (2w, 2w + 1), plus the main input;
    // a coarse level's output (the next level's lowpass) keeps its low-order part as well
    float* outp = base_ptr(B, J.out.b) + J.out.off;
    float* outlp = J.out_lo.b >= 0 ? base_ptr(B, J.out_lo.b) + J.out_lo.off : nullptr;
    for (int i = threadIdx.x; i < (T / 2) * (T / 2); i += blockDim.x) {
        const int p = i / (T / 2), w = i - p * (T / 2);
        const int x = 2 * w;
        const int kb = (p - MLO) * T + x;
        float2 eh = zero2, el = zero2, oh = zero2, ol = zero2;
#pragma unroll
        for (int t = -RS; t <= RS; t++) {
            if ((t & 1) == 0) {
                const int k = kb - (t / 2) * T;
                gacc(eh, el, c2, tap_s<RS>(t), tapl_s<RS>(t), *reinterpret_cast<const float2*>(s_ah + k),
                     *reinterpret_cast<const float2*>(s_al + k));
            } else {
                const int k = kb + ((1 - t) / 2) * T;
                gacc(oh, ol, c2, tap_s<RS>(t), tapl_s<RS>(t), *reinterpret_cast<const float2*>(s_ah + k),
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
            two_sum2(hi, lo);   // the rounded output and its exact remainder
            float* orow = outp + (long long)gy * J.out.rs;
            if (gx < W) orow[gx] = hi.x;
            if (gx + 1 < W) orow[gx + 1] = hi.y;
            if (outlp) {
                float* lrow = outlp + (long long)gy * J.out_lo.rs;
                if (gx < W) lrow[gx] = lo.x;
                if (gx + 1 < W) lrow[gx + 1] = lo.y;
            }
        }
    }
}

// single-precision analysis tile: cout = down(main, fa); out = main - up(cout, fs)
// CENTRED: the tile's staged input is read as x - mu, mu the nearest integer to its
// mean (exact for integer samples, else one rounding of a number no larger than x),
// and the lowpass output gets 2 mu back, exactly the lowpass of the constant mu (the
// 9/7 lowpass has DC gain sqrt(2) per dimension), while the detail of a constant is
// zero.  Rounding errors then scale with the tile's deviation from its mean rather
// than with its values; this is what lets the forward transform's first level, three
// quarters of its LP work, run in plain single precision.
//
// Each of the four passes gives a thread a run of outputs along the filtered
// direction and reads the run's input window once into registers; every output
// still accumulates its taps in the same order as the one-output-per-thread form.

// outputs per thread of a decimating pass over n outputs: the largest of 7, 6, 5 that divides n
constexpr int lp_run_len(int n) { return n % 7 == 0 ? 7 : n % 6 == 0 ? 6 : 5; }

template <int RA, int RS>
struct LevelGeo {
    static constexpr int T = LP_TILE;
    static constexpr int MLO = -(RS / 2);
    static constexpr int MHI = (T - 1 + RS) / 2;
    static constexpr int VN = MHI - MLO + 1;
    static constexpr int MN = 2 * (VN - 1) + 2 * RA + 1;
    static constexpr int Y0 = 2 * MLO - RA;  // main tile origin relative to the output tile origin
    static constexpr int MNS = MN + (MN & 1);   // even row stride: the row pass reads its windows in pairs
    static constexpr int TS = T + 2;            // expanded-row stride: pair stores of 16 rows hit 32 banks
    static constexpr int NA = (MN * VN > VN * TS) ? MN * VN : VN * TS;
    static constexpr int KR = lp_run_len(VN);   // row-pass outputs per thread
    static constexpr int KC = lp_run_len(VN);   // column-pass outputs per thread
    static constexpr int KP = 8;                // expanding passes: output pairs per thread
    static constexpr int SLO = RS / 2, SHI = (RS + 1) / 2;   // an expanded pair reads v[p - SLO .. p + SHI]
    static_assert(VN % KR == 0 && VN % KC == 0 && (T / 2) % KP == 0, "runs tile the passes");
    static_assert(((VN * VN + 3) & ~3) + 32 <= NA, "the synthesis stages cin_lo and the warp sums in s_a");
    // shared memory of one tile, in floats, each array 16-byte aligned
    static constexpr int FLOATS = ((MN * MNS + 3) & ~3) + ((NA + 3) & ~3) + VN * VN;
};

// s_main: MN x MNS floats, s_a: NA, s_v: VN x VN (16-byte aligned); any number of
// threads that is a multiple of 32 (at least 256 for the centring's warp sums: at most
// VN * VN warps)
// SYN: the synthesis tile instead, x = d + up(cin - down(d)) (main = d; cin with its
// low-order part cin_lo where the job has one), CENTRED on mu = half the rounded
// mean of the tile's cin window: e' = (cin - 2 mu) + cin_lo - down(d), x = d + up(e') + mu,
// exact for the real filters because up(2 mu) = mu.
template <int RA, int RS, bool CENTRED, bool SYN = false>
__device__ __forceinline__ void lp_level_tile(const LpJob& J, int tile, const Bases& B, float* s_main, float* s_a,
                                              float* s_v) {
    static_assert(!SYN || CENTRED, "the single-precision synthesis tile is centred");
    using G = LevelGeo<RA, RS>;
    constexpr int T = G::T, MLO = G::MLO, VN = G::VN, MN = G::MN, Y0 = G::Y0, MNS = G::MNS, TS = G::TS;
    const int ty = tile / J.tiles_x, tx = tile - ty * J.tiles_x;
    const int y0 = ty * T, x0 = tx * T;
    const int m0 = y0 / 2, n0 = x0 / 2;
    const int H = J.H, W = J.W, Hh = H / 2, Wh = W / 2;
    const float* mainp = base_ptr(B, J.main.b) + J.main.off;
    const int mrs = J.main.rs;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nwarp = blockDim.x >> 5;

    lp_stage<MN, MNS>(s_main, mainp, mrs, y0 + Y0, x0 + Y0, H, W);
    float mu = 0.f;
    if (SYN) {
        // the tile's cin window (half resolution, periodic) into s_v and its low-order part
        // into s_a, a warp per row: copied asynchronously with the detail, or plainly where
        // they are a tail kernel's resident images; mu from the block sum of the window
        const float* cinp = base_ptr(B, J.cin.b) + J.cin.off;
        const float* cinlp = J.cin_lo.b >= 0 ? base_ptr(B, J.cin_lo.b) + J.cin_lo.off : nullptr;
        const bool cin_sh = __isShared(cinp), lo_sh = cinlp && __isShared(cinlp);
        const int c0 = n0 + MLO;
        const bool inner = c0 >= 0 && c0 + VN <= Wh;
        for (int m = warp; m < VN; m += nwarp) {
            const int gm = wrap_idx(m0 + MLO + m, Hh);
            const float* rowp = cinp + (long long)gm * J.cin.rs;
            const float* lrow = cinlp ? cinlp + (long long)gm * J.cin_lo.rs : nullptr;
            for (int n = lane; n < VN; n += 32) {
                const int gn = inner ? c0 + n : wrap_idx(c0 + n, Wh);
                if (cin_sh) s_v[m * VN + n] = rowp[gn];
                else lp_cp_async4(s_v + m * VN + n, rowp + gn);
                if (lo_sh) s_a[m * VN + n] = lrow[gn];
                else if (cinlp) lp_cp_async4(s_a + m * VN + n, lrow + gn);
            }
        }
        lp_cp_async_wait_all();
        __syncthreads();
        float* s_part = s_a + ((VN * VN + 3) & ~3);   // after the low-order window
        float sum = 0.f;
        for (int i = threadIdx.x; i < VN * VN; i += blockDim.x) sum += s_v[i];
#pragma unroll
        for (int o = 16; o; o >>= 1) sum += __shfl_xor_sync(0xffffffffu, sum, o);
        if (lane == 0) s_part[warp] = sum;
        __syncthreads();
        float tot = 0.f;
        for (int w = 0; w < nwarp; w++) tot += s_part[w];
        mu = rintf(tot / (float)(2 * VN * VN));
        // e' = (cin - 2 mu) + cin_lo, less down(d) in the column pass
        for (int i = threadIdx.x; i < VN * VN; i += blockDim.x) {
            float e = s_v[i] - 2.f * mu;
            if (cinlp) e = e + s_a[i];
            s_v[i] = e;
        }
        __syncthreads();   // s_a is reused below
    } else {
        lp_cp_async_wait_all();
        __syncthreads();
    }
    if (CENTRED && !SYN) {
        // mu: the staged tile's mean, rounded to an integer (a warp per row)
        float sum = 0.f;
        for (int r = warp; r < MN; r += nwarp) {
            const float* row = s_main + r * MNS;
            for (int c = lane; c < MN; c += 32) sum += row[c];
        }
#pragma unroll
        for (int o = 16; o; o >>= 1) sum += __shfl_xor_sync(0xffffffffu, sum, o);
        if (lane == 0) s_v[warp] = sum;
        __syncthreads();
        float tot = 0.f;
        for (int w = 0; w < nwarp; w++) tot += s_v[w];
        mu = rintf(tot / (float)(MN * MN));
        // s_v is next written in the column pass, after the row pass's barrier
    }
    constexpr bool SUB = CENTRED && !SYN;   // the analysis reads its input as x - mu
    // decimating row pass: s_a[r][n] = sum_b fa[b] main[r][2n + RA - b]; a thread takes KR
    // outputs of one row, whose window main[r][2 n0 .. 2 n0 + 2 KR + 2 RA - 2] starts at an
    // even offset (pairs and one more); lanes on consecutive rows
    {
        constexpr int KR = G::KR, NWIN = 2 * KR + 2 * RA - 1;
        for (int i = threadIdx.x; i < MN * (VN / KR); i += blockDim.x) {
            const int run = i / MN, r = i - run * MN;
            const float* w = s_main + r * MNS + 2 * KR * run;
            float x[NWIN];
#pragma unroll
            for (int j = 0; j < NWIN / 2; j++) {
                const float2 pr = *reinterpret_cast<const float2*>(w + 2 * j);
                x[2 * j] = SUB ? pr.x - mu : pr.x;
                x[2 * j + 1] = SUB ? pr.y - mu : pr.y;
            }
            x[NWIN - 1] = SUB ? w[NWIN - 1] - mu : w[NWIN - 1];
            float* dst = s_a + r * VN + KR * run;
#pragma unroll
            for (int k = 0; k < KR; k++) {
                float acc = 0.f;
#pragma unroll
                for (int b = -RA; b <= RA; b++) acc = fmaf(tap_a<RA>(b), x[2 * k + RA - b], acc);
                dst[k] = acc;
            }
        }
    }
    __syncthreads();
    // decimating column pass -> half-resolution values v on [m0+MLO, m0+MHI] x [n0+MLO, n0+MHI];
    // a thread takes KC outputs of one column, lanes on consecutive columns.  The analysis
    // stores the interior 32 x 32 of v, this tile's share of the lowpass output, from here.
    {
        constexpr int KC = G::KC, NWIN = 2 * KC + 2 * RA - 1;
        float* coutp = SYN ? nullptr : base_ptr(B, J.cout.b) + J.cout.off;
        for (int i = threadIdx.x; i < VN * (VN / KC); i += blockDim.x) {
            const int run = i / VN, n = i - run * VN;
            const int mr = KC * run;
            const float* col = s_a + 2 * mr * VN + n;
            float y[NWIN];
#pragma unroll
            for (int j = 0; j < NWIN; j++) y[j] = col[j * VN];
            const int gn = n0 + n + MLO;
            const bool ncol = !SYN && n + MLO >= 0 && n + MLO < T / 2 && gn < Wh;
#pragma unroll
            for (int k = 0; k < KC; k++) {
                float acc = 0.f;
#pragma unroll
                for (int a = -RA; a <= RA; a++) acc = fmaf(tap_a<RA>(a), y[2 * k + RA - a], acc);
                const int m = mr + k;
                if (SYN) {
                    s_v[m * VN + n] = s_v[m * VN + n] - acc;
                } else {
                    s_v[m * VN + n] = acc;
                    const int gm = m0 + m + MLO;
                    if (ncol && m + MLO >= 0 && m + MLO < T / 2 && gm < Hh)
                        coutp[(long long)gm * J.cout.rs + gn] = CENTRED ? acc + 2.f * mu : acc;
                }
            }
        }
    }
    __syncthreads();
    // expanding row pass, by output pairs (x = 2p, 2p + 1):
    //   s_a[m][x] = sum_{t : x - t even} fs[t] v[m][(x - t)/2 - MLO]
    // a thread takes KP pairs of one row (window v[m][p0 - SLO - MLO .. p0 + KP - 1 + SHI - MLO]),
    // lanes on consecutive rows
    constexpr int KP = G::KP, SLO = G::SLO, NWE = KP + G::SLO + G::SHI;
    for (int i = threadIdx.x; i < VN * (T / 2 / KP); i += blockDim.x) {
        const int run = i / VN, m = i - run * VN;
        const int p0 = KP * run;
        const float* vr = s_v + m * VN + p0 - MLO - SLO;
        float z[NWE];
#pragma unroll
        for (int j = 0; j < NWE; j++) z[j] = vr[j];
        float* dst = s_a + m * TS + 2 * p0;
#pragma unroll
        for (int k = 0; k < KP; k++) {
            float ev = 0.f, od = 0.f;
#pragma unroll
            for (int t = -RS; t <= RS; t++) {
                if ((t & 1) == 0) ev = fmaf(tap_s<RS>(t), z[k + SLO - t / 2], ev);        // x = 2p
                else od = fmaf(tap_s<RS>(t), z[k + SLO + (1 - t) / 2], od);                // x = 2p + 1
            }
            *reinterpret_cast<float2*>(dst + 2 * k) = make_float2(ev, od);
        }
    }
    __syncthreads();
    // expanding column pass by output pairs (y = 2p, 2p + 1) and the combination with the main
    // input; a thread takes KP pairs of one column, lanes on consecutive columns
    float* outp = base_ptr(B, J.out.b) + J.out.off;
    for (int i = threadIdx.x; i < T * (T / 2 / KP); i += blockDim.x) {
        const int run = i / T, x = i - run * T;
        const int p0 = KP * run;
        const float* ac = s_a + (p0 - MLO - SLO) * TS + x;
        float z[NWE];
#pragma unroll
        for (int j = 0; j < NWE; j++) z[j] = ac[j * TS];
        const int gx = x0 + x;
        const float* mcol = s_main + (2 * p0 - Y0) * MNS + (x - Y0);
        float* ocol = outp + gx;
#pragma unroll
        for (int k = 0; k < KP; k++) {
            float ev = 0.f, od = 0.f;
#pragma unroll
            for (int t = -RS; t <= RS; t++) {
                if ((t & 1) == 0) ev = fmaf(tap_s<RS>(t), z[k + SLO - t / 2], ev);
                else od = fmaf(tap_s<RS>(t), z[k + SLO + (1 - t) / 2], od);
            }
#pragma unroll
            for (int h = 0; h < 2; h++) {
                const int y = 2 * (p0 + k) + h, gy = y0 + y;
                if (gy < H && gx < W) {
                    const float acc = h ? od : ev;
                    const float mv = mcol[(2 * k + h) * MNS];
                    ocol[(long long)gy * J.out.rs] = SYN ? (mv + acc) + mu : (SUB ? mv - mu : mv) - acc;
                }
            }
        }
    }
}


template <int RA, int RS>
constexpr size_t ff_smem() {
    constexpr int T = LP_TILE;
    constexpr int MLO = -(RS / 2);
    constexpr int MHI = (T - 1 + RS) / 2;
    constexpr int VN = MHI - MLO + 1;
    constexpr int MN = 2 * (VN - 1) + 2 * RA + 1;
    constexpr int NA = (MN * VN > VN * T) ? MN * VN : VN * T;
    constexpr int MNS = MN + (MN & 1), OA = (MN * MNS + 3) & ~3, NA4 = (NA + 3) & ~3;
    return sizeof(float) * (size_t)(OA + 2 * NA4 + 2 * VN * VN + 16);
}

}  // namespace cvc
