// k_dfb.cu -- directional filter bank stages (§2.1), fused tile kernels.
//
// Every stage is a two-channel fan filter bank in ladder form (see
// ct_engine.cu for the lattice reading): one pass over the target coset, one
// over the other, each sample becoming alpha*self + gamma*(16-tap stencil of
// the other coset) with weights betat[a]*betat[b], betat = (-1,-9,9,1)/16.
//
// k_dfb_a: stages 1 and 2 of a detail image in 64 x 64 tiles.  The tile and
//   a 12-sample halo (3 per pass) sit in shared memory as the image's four
//   polyphase planes (the stage-2 channels), so every pass reads unit-stride
//   rows without bank conflicts; the tap tables are compile-time constants;
//   the four passes run in place; the planes are written to the channel
//   arrays, or read from them in the synthesis direction.
// k_dfb_b: one stage s >= 3 of a channel array (a split into even / odd
//   rows).  Rows are staged in shared memory SHEARED by i*q columns (q the
//   parent row), which turns the slope-i stencil (row offset a, column offset
//   -i*a + (b-a)/2) into the same 4 x 4 window for every i; it is evaluated
//   separably, a 4-tap row sum per source sample and a 4-tap sum across rows
//   per target.  Both passes of the stage run in one launch on a 16 x 128
//   tile with a 3-row / 6-column halo.
//
// k_dfb_gsum / k_dfb_g / k_dfb_leaf: the plain path of the longer
//   prototypes (6 or 8 taps), each lifting pass over whole detail images in
//   two launches (diagonal sums, then the targets).
//
// Both directions compute in single precision: the filter-bank weights are
// dyadic and alpha, gamma powers of two, and the inverse's error is dominated
// by the Laplacian-pyramid synthesis, which is compensated (k_lp.cu).
#include "cvc_internal.cuh"

namespace cvc {

__device__ __forceinline__ int wrapd(int a, int n) {
    if ((unsigned)a < (unsigned)n) return a;
    int r = a % n;
    return r < 0 ? r + n : r;
}

// the dyadic taps betat = (-1, -9, 9, 1) / 16 as immediates
constexpr float BT0 = -0.0625f, BT1 = -0.5625f, BT2 = 0.5625f, BT3 = 0.0625f;

// 4-byte asynchronous global -> shared copies: a thread issues all of its
// staging loads before waiting, so a tile's whole halo is in flight at once
__device__ __forceinline__ void cp_async4(float* dst, const float* src) {
    const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(d), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async4s(unsigned dst, const float* src) {
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(dst), "l"(src) : "memory");
}
__device__ __forceinline__ unsigned smem_addr(const float* p) { return (unsigned)__cvta_generic_to_shared(p); }
__device__ __forceinline__ void cp_async_wait_all() {
    asm volatile("cp.async.commit_group;\ncp.async.wait_group 0;\n" ::: "memory");
}

// ============================================================ k_dfb_a
constexpr int SA = DFBA_TILE + 2 * DFBA_HALO;  // 88: tile + halo, image samples
constexpr int PA = SA / 2;                     // 44: polyphase plane side
constexpr int PAS = PA + 1;                    // padded plane row stride

__host__ __device__ constexpr int fdiv2(int a) { return a >= 0 ? a / 2 : -((1 - a) / 2); }
// plane rows (or columns) of parity p whose image index lies in [lo, hi)
__host__ __device__ constexpr int pl0(int lo, int p) { return (lo - p + 1) / 2; }
__host__ __device__ constexpr int pl1(int hi, int p) { return (hi - 1 - p) / 2 + 1; }

// Both stages evaluate their 16-tap stencils separably.
//   Stage 1 (quincunx, taps at ((a+b)/2, (a-b)/2)): the anti-diagonal sums
//     D[p] = sum_m betat[m] x[p + (m, -m)] at the source coset's points, then
//     acc(t) = sum_n betat[n] D[t + (n - 3, n)].
//   Stage 2 (taps at (a, b) in both families): row sums along the target's
//     source plane, then sums down its columns.
// A pass over image-local [lo, hi)^2, lo = 3n, reads the region the previous
// pass left valid, [lo - 3, hi + 3)^2.  Consecutive threads take consecutive
// elements of a region row.

// element offset of plane class (r, c) at plane-local (u, v)
__host__ __device__ constexpr int pofs(int r, int c, int u, int v) { return (2 * r + c) * PA * PAS + u * PAS + v; }

// Visit every (u, v) of [U0, U1) x [V0, V1) with the element offset u*PAS + v:
// thread t owns column V0 + t % NV and walks down rows U0 + t / NV, stepping
// by the number of row chunks, so an access is one running offset plus a
// compile-time displacement.
template <int U0, int U1, int V0, int V1, class F>
__device__ __forceinline__ void region_walk(F&& f) {
    constexpr int NV = V1 - V0, CH = 256 / NV;
    static_assert(NV >= 1 && NV <= 256 && U1 > U0, "region");
    const int t = threadIdx.x;
    if (t >= CH * NV) return;
    const int v = V0 + t % NV;
    int off = (U0 + t / NV) * PAS + v;
    for (int u = U0 + t / NV; u < U1; u += CH, off += CH * PAS) f(off);
}

// stage 1, source class (sr, sc): D[p] = sum_m betat[m] x[p + (m, -m)] over image rows
// [lo-3, hi) and columns [lo, hi+3) of the class, into tmp plane sr
template <int N, bool ODD, int K>
__device__ __forceinline__ void s1_dsum(const float* planes, float* tmp) {
    constexpr int lo = 3 * N, hi = SA - 3 * N;
    constexpr int sr = K, sc = ODD ? K : 1 - K;
    constexpr int o0 = pofs((sr + 0) & 1, (sc - 0) & 1, fdiv2(sr + 0), fdiv2(sc - 0));
    constexpr int o1 = pofs((sr + 1) & 1, (sc - 1) & 1, fdiv2(sr + 1), fdiv2(sc - 1));
    constexpr int o2 = pofs((sr + 2) & 1, (sc - 2) & 1, fdiv2(sr + 2), fdiv2(sc - 2));
    constexpr int o3 = pofs((sr + 3) & 1, (sc - 3) & 1, fdiv2(sr + 3), fdiv2(sc - 3));
    float* D = tmp + sr * PA * PAS;
    region_walk<pl0(lo - 3, sr), pl1(hi, sr), pl0(lo, sc), pl1(hi + 3, sc)>([&](int off) {
        float acc = BT0 * planes[off + o0];
        acc = fmaf(BT1, planes[off + o1], acc);
        acc = fmaf(BT2, planes[off + o2], acc);
        D[off] = fmaf(BT3, planes[off + o3], acc);
    });
}

// stage 1, target class (tr, tc): acc(t) = sum_n betat[n] D[t + (n - 3, n)]
template <int N, bool ODD, int K>
__device__ __forceinline__ void s1_target(float* planes, const float* tmp, float alpha, float gamma) {
    constexpr int lo = 3 * N, hi = SA - 3 * N;
    constexpr int tr = K, tc = ODD ? 1 - K : K;
    constexpr int o0 = ((tr + 1) & 1) * PA * PAS + fdiv2(tr - 3) * PAS + fdiv2(tc + 0);
    constexpr int o1 = ((tr + 2) & 1) * PA * PAS + fdiv2(tr - 2) * PAS + fdiv2(tc + 1);
    constexpr int o2 = ((tr + 3) & 1) * PA * PAS + fdiv2(tr - 1) * PAS + fdiv2(tc + 2);
    constexpr int o3 = ((tr + 4) & 1) * PA * PAS + fdiv2(tr + 0) * PAS + fdiv2(tc + 3);
    float* T = planes + (2 * tr + tc) * PA * PAS;
    region_walk<pl0(lo, tr), pl1(hi, tr), pl0(lo, tc), pl1(hi, tc)>([&](int off) {
        float acc = BT0 * tmp[off + o0];
        acc = fmaf(BT1, tmp[off + o1], acc);
        acc = fmaf(BT2, tmp[off + o2], acc);
        acc = fmaf(BT3, tmp[off + o3], acc);
        T[off] = fmaf(alpha, T[off], gamma * acc);
    });
}

// stage 2, target class (tr, tc) reads class (1-tr, 1-tc) at (u + ky + tr - 2, v + kx + tc - 2):
// row sums into tmp plane tr, then sums down the columns
template <int N, bool ODD, int K>
__device__ __forceinline__ void s2_rowsum(const float* planes, float* tmp) {
    constexpr int lo = 3 * N, hi = SA - 3 * N;
    constexpr int tr = K, tc = ODD ? 1 : 0;
    constexpr int u0 = pl0(lo, tr), u1 = pl1(hi, tr), v0 = pl0(lo, tc), v1 = pl1(hi, tc);
    constexpr int os = (2 * (1 - tr) + (1 - tc)) * PA * PAS + (tc - 2);
    float* Rs = tmp + tr * PA * PAS;
    region_walk<u0 + tr - 2, u1 + tr + 1, v0, v1>([&](int off) {
        float acc = BT0 * planes[off + os];
        acc = fmaf(BT1, planes[off + os + 1], acc);
        acc = fmaf(BT2, planes[off + os + 2], acc);
        Rs[off] = fmaf(BT3, planes[off + os + 3], acc);
    });
}

template <int N, bool ODD, int K>
__device__ __forceinline__ void s2_target(float* planes, const float* tmp, float alpha, float gamma) {
    constexpr int lo = 3 * N, hi = SA - 3 * N;
    constexpr int tr = K, tc = ODD ? 1 : 0;
    constexpr int oh = tr * PA * PAS + (tr - 2) * PAS;
    float* T = planes + (2 * tr + tc) * PA * PAS;
    region_walk<pl0(lo, tr), pl1(hi, tr), pl0(lo, tc), pl1(hi, tc)>([&](int off) {
        float acc = BT0 * tmp[off + oh];
        acc = fmaf(BT1, tmp[off + oh + PAS], acc);
        acc = fmaf(BT2, tmp[off + oh + 2 * PAS], acc);
        acc = fmaf(BT3, tmp[off + oh + 3 * PAS], acc);
        T[off] = fmaf(alpha, T[off], gamma * acc);
    });
}

template <int N, bool ODD>
__device__ __forceinline__ void dfba_stage1(float* planes, float* tmp, float alpha, float gamma) {
    // sources: the even coset {00, 11} for odd targets, {01, 10} for even ones
    s1_dsum<N, ODD, 0>(planes, tmp);
    s1_dsum<N, ODD, 1>(planes, tmp);
    __syncthreads();
    // targets: {01, 10} (odd) or {00, 11}
    s1_target<N, ODD, 0>(planes, tmp, alpha, gamma);
    s1_target<N, ODD, 1>(planes, tmp, alpha, gamma);
    __syncthreads();
}

template <int N, bool ODD>
__device__ __forceinline__ void dfba_stage2(float* planes, float* tmp, float alpha, float gamma) {
    // targets: {11, 01} (odd) or {00, 10}
    s2_rowsum<N, ODD, 0>(planes, tmp);
    s2_rowsum<N, ODD, 1>(planes, tmp);
    __syncthreads();
    s2_target<N, ODD, 0>(planes, tmp, alpha, gamma);
    s2_target<N, ODD, 1>(planes, tmp, alpha, gamma);
    __syncthreads();
}

// the passes of one tile: analysis runs stage 1 then 2, synthesis stage 2 then 1
template <bool SYN, bool FO>
__device__ __forceinline__ void dfba_passes(float* planes, float* tmp, int nst, const PassParams& pp) {
    if (!SYN) {
        dfba_stage1<1, FO>(planes, tmp, pp.a1, pp.g1);
        dfba_stage1<2, !FO>(planes, tmp, pp.a2, pp.g2);
        if (nst == 2) {
            dfba_stage2<3, FO>(planes, tmp, pp.a1, pp.g1);
            dfba_stage2<4, !FO>(planes, tmp, pp.a2, pp.g2);
        }
    } else if (nst == 2) {
        dfba_stage2<1, FO>(planes, tmp, pp.a1, pp.g1);
        dfba_stage2<2, !FO>(planes, tmp, pp.a2, pp.g2);
        dfba_stage1<3, FO>(planes, tmp, pp.a1, pp.g1);
        dfba_stage1<4, !FO>(planes, tmp, pp.a2, pp.g2);
    } else {
        dfba_stage1<1, FO>(planes, tmp, pp.a1, pp.g1);
        dfba_stage1<2, !FO>(planes, tmp, pp.a2, pp.g2);
    }
}

template <bool SYN>
__global__ void __launch_bounds__(256) k_dfb_a(const DfbAJob* __restrict__ jobs, const int* __restrict__ block_job,
                                               Bases B, PassParams pp) {
    __shared__ float planes[4 * PA * PAS];
    __shared__ float tmp[2 * PA * PAS];
    const DfbAJob& J = jobs[block_job[blockIdx.x]];
    const int tile = blockIdx.x - J.first_block;
    const int ty = tile / J.tiles_x, tx = tile - ty * J.tiles_x;
    const int y0 = ty * DFBA_TILE, x0 = tx * DFBA_TILE;
    const int H = J.H, W = J.W, H2 = H / 2, W2 = W / 2;
    // plane-local (u, v) of class (pr, pc) <-> image (y0 - 12 + 2u + pr, x0 - 12 + 2v + pc);
    // class-array index ((y0 - 12)/2 + u, (x0 - 12)/2 + v), periodic in (H/2, W/2)
    const int cu0 = (y0 - DFBA_HALO) / 2, cv0 = (x0 - DFBA_HALO) / 2;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (!SYN) {
        const float* Dp = B.p[J.D.b] + J.D.off;
        const bool inner = x0 - DFBA_HALO >= 0 && x0 - DFBA_HALO + SA <= W;   // no column wrap in this tile
        for (int r = warp; r < SA; r += 8) {
            const float* row = Dp + (long long)wrapd(y0 - DFBA_HALO + r, H) * J.D.rs;
            // image column c of the tile -> plane (r & 1, c & 1), plane column c >> 1
            const unsigned sb = smem_addr(planes + 2 * (r & 1) * PA * PAS + (r >> 1) * PAS);
            for (int c = lane; c < SA; c += 32) {
                const int x = inner ? x0 - DFBA_HALO + c : wrapd(x0 - DFBA_HALO + c, W);
                cp_async4s(sb + 4u * ((c & 1) * PA * PAS + (c >> 1)), row + x);
            }
        }
    } else {
        for (int q = 0; q < 4; q++) {
            const View& V = J.comp[q];
            const float* P = B.p[V.b] + V.off;
            if (V.cs == 1) {
                // row-major channel: plane row u is a run of array row cu
                const bool inner = cv0 >= 0 && cv0 + PA <= W2;
                for (int u = warp; u < PA; u += 8) {
                    const float* row = P + (long long)wrapd(cu0 + u, H2) * V.rs;
                    const unsigned sb = smem_addr(planes + q * PA * PAS + u * PAS);
                    for (int v = lane; v < PA; v += 32)
                        cp_async4s(sb + 4u * v, row + (inner ? cv0 + v : wrapd(cv0 + v, W2)));
                }
            } else {
                // transposed channel (rs = 1): walk along its memory rows, plane column v
                for (int v = warp; v < PA; v += 8) {
                    const float* col = P + (long long)wrapd(cv0 + v, W2) * V.cs;
                    for (int u = lane; u < PA; u += 32)
                        cp_async4s(smem_addr(planes + q * PA * PAS + u * PAS + v), col + wrapd(cu0 + u, H2) * V.rs);
                }
            }
        }
    }
    cp_async_wait_all();
    __syncthreads();
    if (pp.first_odd) dfba_passes<SYN, true>(planes, tmp, J.nst, pp);
    else dfba_passes<SYN, false>(planes, tmp, J.nst, pp);
    // store the 64 x 64 tile: plane-local rows / columns [6, 38)
    constexpr int T2 = DFBA_TILE / 2, H6 = DFBA_HALO / 2;
    if (!SYN) {
        for (int q = 0; q < 4; q++) {
            const View& V = J.comp[q];
            float* P = B.p[V.b] + V.off;
            const bool trans = V.cs != 1;
            for (int k = threadIdx.x; k < T2 * T2; k += blockDim.x) {
                int a = k / T2, b = k - a * T2;
                int u = trans ? b : a, v = trans ? a : b;
                int cu = y0 / 2 + u, cv = x0 / 2 + v;
                if (cu < H2 && cv < W2)
                    P[(long long)cu * V.rs + (long long)cv * V.cs] = planes[q * PA * PAS + (H6 + u) * PAS + H6 + v];
            }
        }
    } else {
        float* Do = B.p[J.D.b] + J.D.off;
        for (int k = threadIdx.x; k < DFBA_TILE * DFBA_TILE; k += blockDim.x) {
            int r = k / DFBA_TILE, c = k - r * DFBA_TILE;
            int y = y0 + r, x = x0 + c;
            if (y < H && x < W) {
                int rr = DFBA_HALO + r, cc = DFBA_HALO + c;
                Do[(long long)y * J.D.rs + x] = planes[(2 * (rr & 1) + (cc & 1)) * PA * PAS + (rr >> 1) * PAS + (cc >> 1)];
            }
        }
    }
}

// ============================================================ k_dfb_b
// Tile frame: RB = 16 + 6 rows (3-row halo) by CB = 116 + 12 columns (6-column
// halo), rows stored with stride CBS = CB + 4.  The coset updated first (F)
// and the second pass's row sums are stored one float to the right of their
// array base, so that every column-pair window below is 8-byte aligned.  A
// thread owns one column pair and one of four interleaved row chunks and walks
// its rows with constant pointer steps; pairs of lanes compute with paired
// FP32 instructions, rounding each lane exactly as the scalar sequence would.
constexpr int RB = DFBB_ROWS + 6, CB = DFBB_COLS + 12, CBS = CB + 4;
constexpr int NPAIR = 64, NCHUNK = 4;   // 256 threads
constexpr int SMB = RB * CBS + 2;       // floats per tile array (room for the shift)
static_assert(CB / 2 <= NPAIR, "one column pair per thread");

__device__ __forceinline__ float2 f2(float a, float b) { return make_float2(a, b); }

// row sums h[rr][x] = sum_b betat[b] S[rr][x + b], rows [SR0, SR1), pairs x = X0 + 2p, p < NP
template <int SR0, int SR1, int X0, int NP>
__device__ __forceinline__ void rowsum_pairs(const float* S, float* H) {
    static_assert(SR0 >= 0 && SR1 <= RB && X0 >= 0 && X0 + 2 * NP + 3 <= CBS, "row-sum window");
    const int p = threadIdx.x & (NPAIR - 1), c = threadIdx.x >> 6;
    if (p >= NP) return;
    const float* s = S + (SR0 + c) * CBS + X0 + 2 * p;
    float* h = H + (SR0 + c) * CBS + X0 + 2 * p;
    for (int rr = SR0 + c; rr < SR1; rr += NCHUNK, s += NCHUNK * CBS, h += NCHUNK * CBS) {
        const float2 a = *reinterpret_cast<const float2*>(s);
        const float2 b = *reinterpret_cast<const float2*>(s + 2);
        const float e = s[4];
        float2 acc = __fmul2_rn(f2(BT0, BT0), a);
        acc = __ffma2_rn(f2(BT1, BT1), f2(a.y, b.x), acc);
        acc = __ffma2_rn(f2(BT2, BT2), b, acc);
        acc = __ffma2_rn(f2(BT3, BT3), f2(b.y, e), acc);
        *reinterpret_cast<float2*>(h) = acc;
    }
}

// targets t[r][x] = alpha t + gamma sum_ia betat[ia] h[r + DB + ia][x - ia], rows [R0, R1),
// pairs x = X0 + 2p, p < NP.  The layout makes the ia-odd pairs 8-byte aligned.
template <int R0, int R1, int X0, int NP, bool ODD>
__device__ __forceinline__ void target_pairs(float* T, const float* H, float alpha, float gamma) {
    constexpr int DB = ODD ? -1 : -2;
    static_assert(R0 + DB >= 0 && R1 + DB + 3 <= RB && X0 >= 3 && X0 + 2 * NP <= CB, "target window");
    const int p = threadIdx.x & (NPAIR - 1), c = threadIdx.x >> 6;
    if (p >= NP) return;
    const float* h = H + (R0 + c + DB) * CBS + X0 + 2 * p;
    float* t = T + (R0 + c) * CBS + X0 + 2 * p;
    const float2 al = f2(alpha, alpha), ga = f2(gamma, gamma);
    for (int r = R0 + c; r < R1; r += NCHUNK, h += NCHUNK * CBS, t += NCHUNK * CBS) {
        const float a0 = h[0], a1 = h[1];                                      // ia = 0: x, x+1
        const float2 b = *reinterpret_cast<const float2*>(h + CBS - 1);        // ia = 1: x-1, x
        const float c0 = h[2 * CBS - 2], c1 = h[2 * CBS - 1];                  // ia = 2: x-2, x-1
        const float2 d = *reinterpret_cast<const float2*>(h + 3 * CBS - 3);    // ia = 3: x-3, x-2
        float2 acc = __fmul2_rn(f2(BT0, BT0), f2(a0, a1));
        acc = __ffma2_rn(f2(BT1, BT1), b, acc);
        acc = __ffma2_rn(f2(BT2, BT2), f2(c0, c1), acc);
        acc = __ffma2_rn(f2(BT3, BT3), d, acc);
        float2 tv = *reinterpret_cast<const float2*>(t);
        tv = __ffma2_rn(al, tv, __fmul2_rn(ga, acc));
        *reinterpret_cast<float2*>(t) = tv;
    }
}

__device__ __forceinline__ int wrap_fast(int v, int C) {
    // v in [0, C + CB): one subtraction when C >= CB, a remainder otherwise
    return v < C ? v : (C >= CB ? v - C : v % C);
}

template <bool SYN>
__global__ void __launch_bounds__(256) k_dfb_b(const DfbBJob* __restrict__ jobs, const int* __restrict__ block_job,
                                               Bases B, PassParams pp) {
    __shared__ __align__(16) float sE[SMB];
    __shared__ __align__(16) float sO[SMB];
    __shared__ __align__(16) float sH[SMB];
    const DfbBJob& J = jobs[block_job[blockIdx.x]];
    const int tile = blockIdx.x - J.first_block;
    const int ty = tile / J.tiles_x, tx = tile - ty * J.tiles_x;
    const int t0 = ty * DFBB_ROWS, c0 = tx * DFBB_COLS;
    const int R2 = J.R2, C = J.C, i = J.i;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nwarp = blockDim.x >> 5;
    const int fo = pp.first_odd;
    // the first-updated coset (odd if fo) sits one float to the right
    float* arr[2] = {sE + (fo ? 0 : 1), sO + (fo ? 1 : 0)};
    // inputs: analysis reads the parent's cosets, synthesis the children.
    // Smem row r <-> coset row t0 - 3 + r; smem column x <-> sheared column c0 - 6 + x,
    // i.e. array column (c0 - 6 + x - i*q) mod C for parent row q = 2*(t0 - 3 + r) + parity
    for (int par = 0; par < 2; par++) {
        const View V = par ? (SYN ? J.c1 : J.po) : (SYN ? J.c0 : J.pe);
        const float* P = B.p[V.b] + V.off;
        float* S = arr[par];
        if (V.cs == 1) {
            for (int r = warp; r < RB; r += nwarp) {
                const int tu = t0 - 3 + r;
                const float* row = P + (long long)wrapd(tu, R2) * V.rs;
                const int vs = wrapd(c0 - 6 - i * (2 * tu + par), C);
                const unsigned sb = smem_addr(S + r * CBS);
                if (vs + CB <= C) {                  // the sheared window does not wrap: no per-element checks
                    const float* src = row + vs;
                    for (int x = lane; x < CB; x += 32) cp_async4s(sb + 4u * x, src + x);
                } else {
                    for (int x = lane; x < CB; x += 32) cp_async4s(sb + 4u * x, row + wrap_fast(vs + x, C));
                }
            }
        } else {
            // transposed array (rows contiguous in memory along t): walk the sheared
            // tile along memory order; for offset w every row r shares the array
            // column v, at tile column x = w + 2*i*r
            const int wlo = i > 0 ? -2 * i * (RB - 1) : 0, whi = CB + (i < 0 ? -2 * i * (RB - 1) : 0);
            const int vbase = c0 - 6 - i * (2 * (t0 - 3) + par);
            for (int k = threadIdx.x; k < (whi - wlo) * RB; k += blockDim.x) {
                const int w = wlo + k / RB, r = k - (k / RB) * RB;
                const int x = w + 2 * i * r;
                if (x < 0 || x >= CB) continue;
                const int v = wrapd(vbase + w, C);
                cp_async4(&S[r * CBS + x], P + (long long)wrapd(t0 - 3 + r, R2) * V.rs + (long long)v * V.cs);
            }
        }
    }
    cp_async_wait_all();
    __syncthreads();
    // pass 1 updates F on columns [3, 125), which covers what pass 2 reads; pass 2
    // updates S on the tile [3, 3 + ROWS) x [6, 122).  Pass-1 row sums sit at the
    // base of sH, pass-2 row sums one float to the right.
    float* F = arr[fo ? 1 : 0];
    float* Sx = arr[fo ? 0 : 1];
    constexpr int NP1 = 61, NH1 = 63, NP2 = 58, NH2 = 60;
    static_assert(3 + 2 * NP1 == CB - 3 && 6 + 2 * NP2 == CB - 6, "pass windows");
    if (fo) {
        rowsum_pairs<0, RB, 0, NH1>(Sx, sH);
        __syncthreads();
        target_pairs<1, DFBB_ROWS + 4, 3, NP1, true>(F, sH, pp.a1, pp.g1);
        __syncthreads();
        rowsum_pairs<1, DFBB_ROWS + 4, 3, NH2>(F, sH + 1);
        __syncthreads();
        target_pairs<3, DFBB_ROWS + 3, 6, NP2, false>(Sx, sH + 1, pp.a2, pp.g2);
    } else {
        rowsum_pairs<0, RB, 0, NH1>(Sx, sH);
        __syncthreads();
        target_pairs<2, DFBB_ROWS + 5, 3, NP1, false>(F, sH, pp.a1, pp.g1);
        __syncthreads();
        rowsum_pairs<2, DFBB_ROWS + 5, 3, NH2>(F, sH + 1);
        __syncthreads();
        target_pairs<3, DFBB_ROWS + 3, 6, NP2, true>(Sx, sH + 1, pp.a2, pp.g2);
    }
    __syncthreads();
    // outputs: analysis writes the children, synthesis the parent's cosets
    const int ncol = min(DFBB_COLS, C - c0);
    for (int par = 0; par < 2; par++) {
        const View V = par ? (SYN ? J.po : J.c1) : (SYN ? J.pe : J.c0);
        float* P = B.p[V.b] + V.off;
        const float* S = arr[par];
        if (V.cs == 1) {
            for (int rr = warp; rr < DFBB_ROWS; rr += nwarp) {
                const int t = t0 + rr;
                if (t >= R2) break;
                float* row = P + (long long)t * V.rs;
                const int vs = wrapd(c0 - i * (2 * t + par), C);
                const float* srow = S + (3 + rr) * CBS + 6;
                if (vs + ncol <= C) {
                    float* dst = row + vs;
                    for (int xx = lane; xx < ncol; xx += 32) dst[xx] = srow[xx];
                } else {
                    for (int xx = lane; xx < ncol; xx += 32) row[wrap_fast(vs + xx, C)] = srow[xx];
                }
            }
        } else {
            // transposed subband: walk along memory order as in the load
            const int wlo = i > 0 ? -2 * i * (DFBB_ROWS - 1) : 0;
            const int whi = DFBB_COLS + (i < 0 ? -2 * i * (DFBB_ROWS - 1) : 0);
            const int vbase = c0 - i * (2 * t0 + par);
            for (int k = threadIdx.x; k < (whi - wlo) * DFBB_ROWS; k += blockDim.x) {
                const int w = wlo + k / DFBB_ROWS, rr = k - (k / DFBB_ROWS) * DFBB_ROWS;
                const int xx = w + 2 * i * rr;
                const int t = t0 + rr;
                if (xx < 0 || xx >= ncol || t >= R2) continue;
                const int v = wrapd(vbase + w, C);
                P[(long long)t * V.rs + (long long)v * V.cs] = S[(3 + rr) * CBS + 6 + xx];
            }
        }
    }
}

// ============================================================ launches
// ============================================================ k_dfb_g
// Longer prototypes: the fan taps sign(a) |beta[a]| of the 6- and 8-tap
// Lagrange half-band interpolators (3, -25, 150, 150, -25, 3)/256 and
// (-5, 49, -245, 1225, 1225, -245, 49, -5)/2048 at odd a (dyadic: exact).
__constant__ float c_fan6[6] = {-3.f / 256, -25.f / 256, -150.f / 256, 150.f / 256, 25.f / 256, 3.f / 256};
__constant__ float c_fan8[8] = {-5.f / 2048, -49.f / 2048, -245.f / 2048, -1225.f / 2048,
                                1225.f / 2048, 245.f / 2048, 49.f / 2048, 5.f / 2048};

// a channel of the tree: origin, family (0: c, 1: r) and slope index
struct GChan {
    int o_r, o_c, T, i;
};

__device__ __forceinline__ void g_basis(int s, const GChan& ch, int b[4]) {
    if (s == 1) {
        b[0] = 1; b[1] = 0; b[2] = 0; b[3] = 1;
    } else if (s == 2) {
        b[0] = 1; b[1] = 1;
        b[2] = ch.T == 0 ? 1 : -1;
        b[3] = ch.T == 0 ? -1 : 1;
    } else {
        const int q = 1 << (s - 2), i = ch.i;
        if (ch.T == 0) { b[0] = q; b[1] = -2 * i; b[2] = q; b[3] = -2 * i - 2; }
        else { b[0] = -2 * i; b[1] = q; b[2] = -2 * i - 2; b[3] = q; }
    }
}

// Follow sample (r, c) down the tree through stages 1..s: on return ch is its
// stage-s channel, b that channel's basis, and the result its parity there.
// With descend, the walk also steps into the stage-s child (the leaf for s = k)
// and *cid is the child's index in tree order.  The lattice coordinates are
// (adj(B) (r - o)) / det B with |det B| = 2^(st-1); only their parity is
// needed, so the exact divisions are shifts and the sign of det is dropped.
__device__ __forceinline__ int g_walk(int r, int c, int s, bool descend, GChan& ch, int b[4], int* cid) {
    ch = GChan{0, 0, 0, 0};
    int id = 0, par = 0;
    for (int st = 1; st <= s; st++) {
        g_basis(st, ch, b);
        const int dr = r - ch.o_r, dc = c - ch.o_c;
        par = (((b[3] * dr - b[2] * dc) >> (st - 1)) + ((b[0] * dc - b[1] * dr) >> (st - 1))) & 1;
        if (st == s && !descend) break;
        id = 2 * id + par;
        if (par) {
            ch.o_r += b[0];
            ch.o_c += b[1];
        }
        if (st == 1) { ch.T = par; ch.i = 0; }
        else if (st == 2) ch.i = par ? 0 : -1;
        else ch.i = 2 * ch.i + par;
    }
    if (cid) *cid = id;
    return par;
}

// The stage-s channel of a sample (its family, slope index and parity) depends
// on (r, c) alone and repeats with period P_s = 2^(s-1) (2 for s = 1): every
// stage-s channel lattice contains P_s Z^2 and has a power-of-two index.  The
// patterns of stages 1..6 are generated at compile time (the walk above, on
// the host) into one table of 16-bit entries parity | family << 1 |
// (slope + 32) << 2, so that the passes look a sample's channel up.
__host__ __device__ constexpr int g_period(int s) { return s == 1 ? 2 : 1 << (s - 1); }
__host__ __device__ constexpr int g_tab_off(int s) {
    int o = 0;
    for (int t = 1; t < s; t++) o += g_period(t) * g_period(t);
    return o;
}
constexpr int G_TAB_N = g_tab_off(CVC_MAX_DIRS_LOG2 + 1);
struct GTab {
    uint16_t v[G_TAB_N];
};
constexpr GTab g_make_tab() {
    GTab t{};
    for (int s = 1; s <= CVC_MAX_DIRS_LOG2; s++) {
        const int P = g_period(s);
        for (int r = 0; r < P; r++)
            for (int c = 0; c < P; c++) {
                int o_r = 0, o_c = 0, T = 0, i = 0, par = 0;
                for (int st = 1; st <= s; st++) {
                    int b0 = 1, b1 = 0, b2 = 0, b3 = 1;
                    if (st == 2) {
                        b1 = 1;
                        b2 = T == 0 ? 1 : -1;
                        b3 = T == 0 ? -1 : 1;
                    } else if (st >= 3) {
                        const int q = 1 << (st - 2);
                        if (T == 0) { b0 = q; b1 = -2 * i; b2 = q; b3 = -2 * i - 2; }
                        else { b0 = -2 * i; b1 = q; b2 = -2 * i - 2; b3 = q; }
                    }
                    const int det = b0 * b3 - b1 * b2, dr = r - o_r, dc = c - o_c;
                    par = ((b3 * dr - b2 * dc) / det + (b0 * dc - b1 * dr) / det) & 1;
                    if (st == s) break;
                    if (par) { o_r += b0; o_c += b1; }
                    if (st == 1) { T = par; i = 0; }
                    else if (st == 2) i = par ? 0 : -1;
                    else i = 2 * i + par;
                }
                t.v[g_tab_off(s) + r * P + c] = (uint16_t)(par | (T << 1) | ((i + 32) << 2));
            }
    }
    return t;
}
__device__ const GTab c_gtab = g_make_tab();

// channel of sample (r, c) at stage s from the table: its basis, and its parity
__device__ __forceinline__ int g_lookup(int r, int c, int s, int b[4]) {
    const int P = g_period(s);
    const unsigned e = __ldg(&c_gtab.v[g_tab_off(s) + (r & (P - 1)) * P + (c & (P - 1))]);
    g_basis(s, GChan{0, 0, (int)((e >> 1) & 1), (int)(e >> 2) - 32}, b);
    return (int)(e & 1);
}

// A lifting pass of stage s makes every sample t of parity `target`
//   alpha * x[t] + gamma * sum_{a,b} bt[a] bt[b] x[t + delta(a,b)],
// delta(a,b) = ((a+b)/2) B1 + ((a-b)/2) B2 (B1, B2 the channel's basis).  With
// u = (b+1)/2 the offset is ((a-1)/2) B1 + ((a+1)/2) B2 + u (B1 - B2), so the
// sum splits into diagonal sums at the other parity,
//   S[p] = sum_u bt[2u-1] x[p + u (B1 - B2)]                 (k_dfb_gsum)
// and a sum of n of them per target,
//   acc(t) = sum_a bt[a] S[t + ((a-1)/2) B1 + ((a+1)/2) B2]   (k_dfb_g):
// 2n loads per target instead of n^2.  S lives in the level's spare buffer.
__global__ void __launch_bounds__(256) k_dfb_gsum(const DfbGJob* __restrict__ jobs,
                                                  const int* __restrict__ block_job, int s, int target,
                                                  Bases bases) {
    const DfbGJob& J = jobs[block_job[blockIdx.x]];
    const long long pix = (long long)(blockIdx.x - J.first_block) * 256 + threadIdx.x;
    if (s > J.k || pix >= (long long)J.H * J.W) return;
    const int r = (int)(pix / J.W), c = (int)(pix % J.W);
    int b[4];
    if (g_lookup(r, c, s, b) == target) return;                        // sums sit at the other parity
    const float* D = bases.p[J.D.b] + J.D.off;
    const int n = J.ntaps, h = n / 2;
    const float* bt = n == 6 ? c_fan6 : c_fan8;
    const int er = b[0] - b[2], ec = b[1] - b[3];                      // B1 - B2
    float acc = 0.f;
    for (int u = 1 - h; u <= h; u++) {
        const int rr = wrapd(r + u * er, J.H), cc = wrapd(c + u * ec, J.W);
        acc = fmaf(bt[u - 1 + h], D[(long long)rr * J.D.rs + cc], acc);   // tap b = 2u - 1
    }
    bases.p[J.T.b][J.T.off + (long long)r * J.T.rs + c] = acc;
}

__global__ void __launch_bounds__(256) k_dfb_g(const DfbGJob* __restrict__ jobs, const int* __restrict__ block_job,
                                               int s, int target, float alpha, float gamma, Bases bases) {
    const DfbGJob& J = jobs[block_job[blockIdx.x]];
    const long long pix = (long long)(blockIdx.x - J.first_block) * 256 + threadIdx.x;
    if (s > J.k || pix >= (long long)J.H * J.W) return;
    const int r = (int)(pix / J.W), c = (int)(pix % J.W);
    int b[4];
    if (g_lookup(r, c, s, b) != target) return;
    const float* S = bases.p[J.T.b] + J.T.off;
    const int n = J.ntaps;
    const float* bt = n == 6 ? c_fan6 : c_fan8;
    float acc = 0.f;
    for (int ia = 0; ia < n; ia++) {
        const int a = 2 * ia - (n - 1), d1 = (a - 1) / 2, d2 = (a + 1) / 2;     // exact: a is odd
        const int rr = wrapd(r + d1 * b[0] + d2 * b[2], J.H), cc = wrapd(c + d1 * b[1] + d2 * b[3], J.W);
        acc = fmaf(bt[ia], S[(long long)rr * J.T.rs + cc], acc);
    }
    float* x = bases.p[J.D.b] + J.D.off + (long long)r * J.D.rs + c;
    *x = fmaf(alpha, *x, gamma * acc);
}

// copy between the detail image and the level's subbands (tree order, each
// on its rectangular lattice: family c 2^(k-1) x 2, family r 2 x 2^(k-1); k = 1
// the two row-compacted quincunx halves); to_layout: image -> subbands
__global__ void __launch_bounds__(256) k_dfb_leaf(const DfbGJob* __restrict__ jobs,
                                                  const int* __restrict__ block_job, int to_layout, Bases bases) {
    const DfbGJob& J = jobs[block_job[blockIdx.x]];
    const long long pix = (long long)(blockIdx.x - J.first_block) * 256 + threadIdx.x;
    if (pix >= (long long)J.H * J.W) return;
    const int r = (int)(pix / J.W), c = (int)(pix % J.W), k = J.k;
    GChan ch;
    int b[4], cid;
    g_walk(r, c, k, true, ch, b, &cid);
    int a, bc, w;
    if (k == 1) {
        a = r;
        bc = c >> 1;
        w = J.W / 2;
    } else {
        const int R = ch.T == 0 ? (1 << (k - 1)) : 2, C = ch.T == 0 ? 2 : (1 << (k - 1));
        a = (r - wrapd(ch.o_r, R)) / R;
        bc = (c - wrapd(ch.o_c, C)) / C;
        w = J.W / C;
    }
    float* coef = bases.p[B_COEF] + J.slot0 + (long long)cid * (((long long)J.H * J.W) >> k) + (long long)a * w + bc;
    float* x = bases.p[J.D.b] + J.D.off + (long long)r * J.D.rs + c;
    if (to_layout) *coef = *x;
    else *x = *coef;
}

PassParams pass_params(Mode m) {
    switch (m) {
        case FWD: return {1, 0.5f, -0.5f, 1.f, 1.f};       // predict odd, update even
        case INV_ADJ: return {0, 1.f, 1.f, 2.f, -1.f};     // transpose of the inverse stage
        case INV: return {0, 1.f, -1.f, 2.f, 1.f};         // undo update, undo predict
        default: return {1, 0.5f, 0.5f, 1.f, -1.f};        // FWD_ADJ: transpose of the forward stage
    }
}

cudaError_t launch_dfb(const LaunchDfb& L, Mode m, Bases bases, cudaStream_t st) {
    if (L.nblocks == 0) return cudaSuccess;
    const bool syn = (m == INV || m == FWD_ADJ);
    const PassParams pp = pass_params(m);
    if (L.kind == 0) {
        const DfbAJob* j = static_cast<const DfbAJob*>(L.d_jobs);
        if (syn) k_dfb_a<true><<<L.nblocks, 256, 0, st>>>(j, L.d_block_job, bases, pp);
        else k_dfb_a<false><<<L.nblocks, 256, 0, st>>>(j, L.d_block_job, bases, pp);
    } else if (L.kind == 1) {
        const DfbBJob* j = static_cast<const DfbBJob*>(L.d_jobs);
        if (syn) k_dfb_b<true><<<L.nblocks, 256, 0, st>>>(j, L.d_block_job, bases, pp);
        else k_dfb_b<false><<<L.nblocks, 256, 0, st>>>(j, L.d_block_job, bases, pp);
    } else if (L.kind == 2) {
        k_dfb_gsum<<<L.nblocks, 256, 0, st>>>(static_cast<const DfbGJob*>(L.d_jobs), L.d_block_job, L.s, L.target,
                                              bases);
    } else if (L.kind == 4) {
        k_dfb_g<<<L.nblocks, 256, 0, st>>>(static_cast<const DfbGJob*>(L.d_jobs), L.d_block_job, L.s, L.target,
                                           L.alpha, L.gamma, bases);
    } else {
        k_dfb_leaf<<<L.nblocks, 256, 0, st>>>(static_cast<const DfbGJob*>(L.d_jobs), L.d_block_job, L.target,
                                              bases);
    }
    return cudaGetLastError();
}

}  // namespace cvc
