// dfb_tile.cuh -- the directional filter bank tiles (§2.1) as device
// functions, shared by the per-stage kernels (k_dfb.cu) and the tail kernel
// that runs a plane's coarse levels in one block (k_tail.cu).
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
//
// A tile's input may live in global memory (asynchronous copies) or, inside
// the tail kernel, in shared memory (plain copies); every output element is
// computed by the same sequence of operations either way.
#pragma once
#include "cvc_internal.cuh"

namespace cvc {

// a mod n in [0, n); indices at most one period outside take no division
__device__ __forceinline__ int wrapd(int a, int n) {
    if ((unsigned)a < (unsigned)n) return a;
    const int b = a < 0 ? a + n : a - n;
    if ((unsigned)b < (unsigned)n) return b;
    const int r = a % n;
    return r < 0 ? r + n : r;
}

// the fan taps sign(a) |beta[a]| of the NT-tap prototype, a = 2t - (NT - 1), as
// compile-time immediates: NT = 4, (-1, 9, 9, -1)/16; NT = 6 and 8, the longer
// Lagrange half-band interpolators (3, -25, 150, 150, -25, 3)/256 and
// (-5, 49, -245, 1225, 1225, -245, 49, -5)/2048 (all dyadic: exact)
__host__ __device__ constexpr float fan_tap(int NT, int t) {
    return NT == 4 ? (t == 0 ? -1.f : t == 1 ? -9.f : t == 2 ? 9.f : 1.f) / 16.f
         : NT == 6 ? (t == 0 ? -3.f : t == 1 ? -25.f : t == 2 ? -150.f : t == 3 ? 150.f : t == 4 ? 25.f : 3.f) / 256.f
                   : (t == 0 ? -5.f : t == 1 ? -49.f : t == 2 ? -245.f : t == 3 ? -1225.f
                      : t == 4 ? 1225.f : t == 5 ? 245.f : t == 6 ? 49.f : 5.f) / 2048.f;
}

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
// Geometry of the NT-tap tiles: one pass reaches R = NT - 1 samples, the four
// passes of stages 1 and 2 need a halo of 4R around the 64 x 64 tile.
template <int NT>
struct AGeo {
    static constexpr int R = NT - 1;
    static constexpr int HALO = 4 * R;                   // 12, 20, 28
    static constexpr int SA = DFBA_TILE + 2 * HALO;      // tile + halo, image samples
    static constexpr int PA = SA / 2;                    // polyphase plane side
    static constexpr int PAS = PA + 1;                   // padded plane row stride
    static constexpr int SMEM = 6 * PA * PAS * 4;        // four planes and two scratch planes (bytes)
};
static_assert(AGeo<4>::HALO == DFBA_HALO, "4-tap halo");

__host__ __device__ constexpr int fdiv2(int a) { return a >= 0 ? a / 2 : -((1 - a) / 2); }
// plane rows (or columns) of parity p whose image index lies in [lo, hi)
__host__ __device__ constexpr int pl0(int lo, int p) { return (lo - p + 1) / 2; }
__host__ __device__ constexpr int pl1(int hi, int p) { return (hi - 1 - p) / 2 + 1; }

// Both stages evaluate their NT x NT stencils separably.
//   Stage 1 (quincunx, taps at ((a+b)/2, (a-b)/2)): the anti-diagonal sums
//     D[p] = sum_m bt[m] x[p + (m, -m)] at the source coset's points, then
//     acc(t) = sum_n bt[n] D[t + (n - R, n)].
//   Stage 2 (taps at (a, b) in both families): row sums along the target's
//     source plane, then sums down its columns, the row sums kept in registers.
// A pass over image-local [lo, hi)^2, lo = R n, reads the region the previous
// pass left valid, [lo - R, hi + R)^2.  Consecutive threads take consecutive
// elements of a region row.

// element offset of plane class (r, c) at plane-local (u, v)
template <int NT>
__host__ __device__ constexpr int pofs(int r, int c, int u, int v) {
    return (2 * r + c) * AGeo<NT>::PA * AGeo<NT>::PAS + u * AGeo<NT>::PAS + v;
}

// Visit every (u, v) of [U0, U1) x [V0, V1) with the element offset u*PAS + v:
// thread t owns column V0 + t % NV and walks down rows U0 + t / NV, stepping
// by the number of row chunks, so an access is one running offset plus a
// compile-time displacement.
template <int NT, int U0, int U1, int V0, int V1, class F>
__device__ __forceinline__ void region_walk(F&& f) {
    constexpr int NV = V1 - V0, CH = 256 / NV, PAS = AGeo<NT>::PAS;
    static_assert(NV >= 1 && NV <= 256 && U1 > U0, "region");
    static_assert(U0 >= 0 && V0 >= 0 && U1 <= AGeo<NT>::PA && V1 <= AGeo<NT>::PA, "region inside the planes");
    const int t = threadIdx.x;
    if (t >= CH * NV) return;
    const int v = V0 + t % NV;
    int off = (U0 + t / NV) * PAS + v;
    for (int u = U0 + t / NV; u < U1; u += CH, off += CH * PAS) f(off);
}

// stage 1, source class (sr, sc): D[p] = sum_m bt[m] x[p + (m, -m)] over image rows
// [lo-R, hi) and columns [lo, hi+R) of the class, into tmp plane sr
template <int NT, int N, bool ODD, int K>
__device__ __forceinline__ void s1_dsum(const float* planes, float* tmp) {
    using G = AGeo<NT>;
    constexpr int lo = G::R * N, hi = G::SA - G::R * N;
    constexpr int sr = K, sc = ODD ? K : 1 - K;
    float* D = tmp + sr * G::PA * G::PAS;
    region_walk<NT, pl0(lo - G::R, sr), pl1(hi, sr), pl0(lo, sc), pl1(hi + G::R, sc)>([&](int off) {
        float acc = fan_tap(NT, 0) * planes[off + pofs<NT>(sr & 1, sc & 1, fdiv2(sr), fdiv2(sc))];
#pragma unroll
        for (int m = 1; m < NT; m++)
            acc = fmaf(fan_tap(NT, m), planes[off + pofs<NT>((sr + m) & 1, (sc - m) & 1, fdiv2(sr + m), fdiv2(sc - m))],
                       acc);
        D[off] = acc;
    });
}

// stage 1, target class (tr, tc): acc(t) = sum_n bt[n] D[t + (n - R, n)]
template <int NT, int N, bool ODD, int K>
__device__ __forceinline__ void s1_target(float* planes, const float* tmp, float alpha, float gamma) {
    using G = AGeo<NT>;
    constexpr int lo = G::R * N, hi = G::SA - G::R * N;
    constexpr int tr = K, tc = ODD ? 1 - K : K;
    float* T = planes + (2 * tr + tc) * G::PA * G::PAS;
    region_walk<NT, pl0(lo, tr), pl1(hi, tr), pl0(lo, tc), pl1(hi, tc)>([&](int off) {
        float acc = 0.f;
#pragma unroll
        for (int n = 0; n < NT; n++) {
            const int o = ((tr - G::R + n) & 1) * G::PA * G::PAS + fdiv2(tr - G::R + n) * G::PAS + fdiv2(tc + n);
            acc = n == 0 ? fan_tap(NT, 0) * tmp[off + o] : fmaf(fan_tap(NT, n), tmp[off + o], acc);
        }
        T[off] = fmaf(alpha, T[off], gamma * acc);
    });
}

template <int NT, int N, bool ODD>
__device__ __forceinline__ void dfba_stage1(float* planes, float* tmp, float alpha, float gamma) {
    // sources: the even coset {00, 11} for odd targets, {01, 10} for even ones
    s1_dsum<NT, N, ODD, 0>(planes, tmp);
    s1_dsum<NT, N, ODD, 1>(planes, tmp);
    __syncthreads();
    // targets: {01, 10} (odd) or {00, 11}
    s1_target<NT, N, ODD, 0>(planes, tmp, alpha, gamma);
    s1_target<NT, N, ODD, 1>(planes, tmp, alpha, gamma);
    __syncthreads();
}

// stage 2, target class (tr, tc), which reads class (1-tr, 1-tc) at
// (u + ky + tr - NT/2, v + kx + tc - NT/2), with the row sums kept in
// registers: thread t owns column v of the target region and a run of L
// consecutive rows; it forms each source row sum once (the NT - 1 rows above
// its run once more) and keeps the NT its current target needs, so nothing
// goes through the scratch planes.  Each row sum accumulates its taps in kx
// order and each target its row sums in ky order, as a staged evaluation does.
template <int NT>
__device__ __forceinline__ float s2_row(const float* p) {
    float acc = fan_tap(NT, 0) * p[0];
#pragma unroll
    for (int kx = 1; kx < NT; kx++) acc = fmaf(fan_tap(NT, kx), p[kx], acc);
    return acc;
}

template <int NT, int N, bool ODD, int K>
__device__ __forceinline__ void s2_fused(float* planes, float alpha, float gamma) {
    using G = AGeo<NT>;
    constexpr int lo = G::R * N, hi = G::SA - G::R * N;
    constexpr int tr = K, tc = ODD ? 1 : 0;
    constexpr int u0 = pl0(lo, tr), u1 = pl1(hi, tr), v0 = pl0(lo, tc), v1 = pl1(hi, tc);
    constexpr int NV = v1 - v0, NU = u1 - u0, S = 256 / NV, L = (NU + S - 1) / S;
    constexpr int PAS = G::PAS, PL = G::PA * G::PAS;
    // source rows u0 + tr - NT/2 .. u1 + tr - NT/2 + NT - 2, columns v0 + tc - NT/2 .. v1 + tc - NT/2 + NT - 2
    static_assert(u0 + tr - NT / 2 >= 0 && u1 + tr - NT / 2 + NT - 1 <= G::PA, "source rows inside the plane");
    static_assert(v0 + tc - NT / 2 >= 0 && v1 + tc - NT / 2 + NT - 1 <= G::PA, "source columns inside the plane");
    static_assert(NV >= 1 && NV <= 256 && S * L >= NU, "runs cover the region");
    const int t = threadIdx.x;
    if (t >= S * NV) return;
    const int v = v0 + t % NV;
    const int ua = u0 + (t / NV) * L, ub = min(ua + L, u1);
    if (ua >= ub) return;
    float* T = planes + (2 * tr + tc) * PL + ua * PAS + v;
    const float* src = planes + (2 * (1 - tr) + (1 - tc)) * PL + (ua + tr - NT / 2) * PAS + v + tc - NT / 2;
    const int cnt = ub - ua;
    float w[L + NT - 1];   // w[j]: row sum of source row ua + tr - NT/2 + j
#pragma unroll
    for (int j = 0; j < NT - 1; j++) w[j] = s2_row<NT>(src + j * PAS);
#pragma unroll
    for (int k = 0; k < L; k++) {
        if (k < cnt) {
            w[k + NT - 1] = s2_row<NT>(src + (k + NT - 1) * PAS);
            float acc = fan_tap(NT, 0) * w[k];
#pragma unroll
            for (int ky = 1; ky < NT; ky++) acc = fmaf(fan_tap(NT, ky), w[k + ky], acc);
            T[k * PAS] = fmaf(alpha, T[k * PAS], gamma * acc);
        }
    }
}

template <int NT, int N, bool ODD>
__device__ __forceinline__ void dfba_stage2(float* planes, float alpha, float gamma) {
    // targets: {11, 01} (odd) or {00, 10}; each reads only the other class of its row parity
    s2_fused<NT, N, ODD, 0>(planes, alpha, gamma);
    s2_fused<NT, N, ODD, 1>(planes, alpha, gamma);
    __syncthreads();
}

// the passes of one tile: analysis runs stage 1 then 2, synthesis stage 2 then 1
template <int NT, bool SYN, bool FO>
__device__ __forceinline__ void dfba_passes(float* planes, float* tmp, int nst, const PassParams& pp) {
    if (!SYN) {
        dfba_stage1<NT, 1, FO>(planes, tmp, pp.a1, pp.g1);
        dfba_stage1<NT, 2, !FO>(planes, tmp, pp.a2, pp.g2);
        if (nst == 2) {
            dfba_stage2<NT, 3, FO>(planes, pp.a1, pp.g1);
            dfba_stage2<NT, 4, !FO>(planes, pp.a2, pp.g2);
        }
    } else if (nst == 2) {
        dfba_stage2<NT, 1, FO>(planes, pp.a1, pp.g1);
        dfba_stage2<NT, 2, !FO>(planes, pp.a2, pp.g2);
        dfba_stage1<NT, 3, FO>(planes, tmp, pp.a1, pp.g1);
        dfba_stage1<NT, 4, !FO>(planes, tmp, pp.a2, pp.g2);
    } else {
        dfba_stage1<NT, 1, FO>(planes, tmp, pp.a1, pp.g1);
        dfba_stage1<NT, 2, !FO>(planes, tmp, pp.a2, pp.g2);
    }
}


// one 64 x 64 tile of stages 1 and 2 (smem_a: AGeo<NT>::SMEM bytes of shared memory)
template <bool SYN, int NT>
__device__ __forceinline__ void dfb_a_tile(const DfbAJob& J, int tile, const Bases& B, const PassParams& pp,
                                           float* smem_a) {
    using G = AGeo<NT>;
    constexpr int SA = G::SA, PA = G::PA, PAS = G::PAS, HALO = G::HALO, PL = PA * PAS;
    static_assert(HALO % 4 == 0 && DFBA_TILE % 4 == 0, "a tile's halo starts on a 16-byte column boundary");
    static_assert(SA / 4 <= 32 && PA / 2 <= 32 && DFBA_TILE / 2 == 32, "one lane per vector of a row");
    float* planes = smem_a;
    float* tmp = smem_a + 4 * PL;
    const int ty = tile / J.tiles_x, tx = tile - ty * J.tiles_x;
    const int y0 = ty * DFBA_TILE, x0 = tx * DFBA_TILE;
    const int H = J.H, W = J.W, H2 = H / 2, W2 = W / 2;
    // plane-local (u, v) of class (pr, pc) <-> image (y0 - HALO + 2u + pr, x0 - HALO + 2v + pc);
    // class-array index ((y0 - HALO)/2 + u, (x0 - HALO)/2 + v), periodic in (H/2, W/2)
    const int cu0 = (y0 - HALO) / 2, cv0 = (x0 - HALO) / 2;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (!SYN) {
        const float* Dp = base_ptr(B, J.D.b) + J.D.off;
        const bool inner = x0 - HALO >= 0 && x0 - HALO + SA <= W;   // no column wrap in this tile
        if (__isShared(Dp)) {
            // a tail kernel's resident detail image: plain copies
            for (int r = warp; r < SA; r += 8) {
                const float* row = Dp + (long long)wrapd(y0 - HALO + r, H) * J.D.rs;
                float* pr = planes + 2 * (r & 1) * PL + (r >> 1) * PAS;
                for (int c = lane; c < SA; c += 32) pr[(c & 1) * PL + (c >> 1)] = row[wrapd(x0 - HALO + c, W)];
            }
        } else if (inner && (reinterpret_cast<uintptr_t>(Dp) & 15) == 0 && (J.D.rs & 3) == 0) {
            // 16-byte loads: lane k < SA/4 takes image columns 4k .. 4k+3 of a row, i.e. plane
            // columns 2k, 2k+1 of the row's two planes; a warp has half of its rows in flight at once
            constexpr int RPW = (SA + 7) / 8, NB = (RPW + 1) / 2;
            const float* base = Dp + (x0 - HALO) + 4 * lane;
#pragma unroll
            for (int h = 0; h < 2; h++) {
                float4 v[NB];
#pragma unroll
                for (int b = 0; b < NB; b++) {
                    const int r = warp + 8 * (h * NB + b);
                    if (r < SA && lane < SA / 4)
                        v[b] = *reinterpret_cast<const float4*>(base + (long long)wrapd(y0 - HALO + r, H) * J.D.rs);
                }
#pragma unroll
                for (int b = 0; b < NB; b++) {
                    const int r = warp + 8 * (h * NB + b);
                    if (r < SA && lane < SA / 4) {
                        float* p = planes + 2 * (r & 1) * PL + (r >> 1) * PAS + 2 * lane;
                        p[0] = v[b].x;
                        p[PL] = v[b].y;
                        p[1] = v[b].z;
                        p[PL + 1] = v[b].w;
                    }
                }
            }
        } else {
            for (int r = warp; r < SA; r += 8) {
                const float* row = Dp + (long long)wrapd(y0 - HALO + r, H) * J.D.rs;
                // image column c of the tile -> plane (r & 1, c & 1), plane column c >> 1
                const unsigned sb = smem_addr(planes + 2 * (r & 1) * PL + (r >> 1) * PAS);
                for (int c = lane; c < SA; c += 32) {
                    const int x = inner ? x0 - HALO + c : wrapd(x0 - HALO + c, W);
                    cp_async4s(sb + 4u * ((c & 1) * PL + (c >> 1)), row + x);
                }
            }
        }
    } else {
        const bool inner = cu0 >= 0 && cu0 + PA <= H2 && cv0 >= 0 && cv0 + PA <= W2;   // no wrap in this tile
        constexpr int RPW = (PA + 7) / 8;
        for (int q = 0; q < 4; q++) {
            const View& V = J.comp[q];
            const float* P = base_ptr(B, V.b) + V.off;
            float* pl = planes + q * PL;
            const bool al8 = (reinterpret_cast<uintptr_t>(P) & 7) == 0;
            if (__isShared(P)) {
                // a tail kernel's resident channel array: plain copies
                for (int u = warp; u < PA; u += 8)
                    for (int v = lane; v < PA; v += 32)
                        pl[u * PAS + v] = P[(long long)wrapd(cu0 + u, H2) * V.rs + (long long)wrapd(cv0 + v, W2) * V.cs];
            } else if (V.cs == 1 && inner && al8 && (V.rs & 1) == 0) {
                // row-major channel, 8-byte loads: lane k < PA/2 takes plane columns 2k, 2k+1 of
                // plane row u = warp + 8b (cv0 is even)
                const float* base = P + (long long)cu0 * V.rs + cv0 + 2 * lane;
                float2 v[RPW];
#pragma unroll
                for (int b = 0; b < RPW; b++) {
                    const int u = warp + 8 * b;
                    if (u < PA && lane < PA / 2) v[b] = *reinterpret_cast<const float2*>(base + (long long)u * V.rs);
                }
#pragma unroll
                for (int b = 0; b < RPW; b++) {
                    const int u = warp + 8 * b;
                    if (u < PA && lane < PA / 2) {
                        pl[u * PAS + 2 * lane] = v[b].x;
                        pl[u * PAS + 2 * lane + 1] = v[b].y;
                    }
                }
            } else if (V.rs == 1 && inner && al8 && (V.cs & 1) == 0) {
                // transposed channel (contiguous along u), 8-byte loads: lane k < PA/2 takes plane
                // rows 2k, 2k+1 of plane column v = warp + 8b (cu0 is even)
                const float* base = P + cu0 + 2 * lane + (long long)cv0 * V.cs;
                float2 w[RPW];
#pragma unroll
                for (int b = 0; b < RPW; b++) {
                    const int v = warp + 8 * b;
                    if (v < PA && lane < PA / 2) w[b] = *reinterpret_cast<const float2*>(base + (long long)v * V.cs);
                }
#pragma unroll
                for (int b = 0; b < RPW; b++) {
                    const int v = warp + 8 * b;
                    if (v < PA && lane < PA / 2) {
                        pl[2 * lane * PAS + v] = w[b].x;
                        pl[(2 * lane + 1) * PAS + v] = w[b].y;
                    }
                }
            } else if (V.cs == 1) {
                // row-major channel: plane row u is a run of array row cu
                for (int u = warp; u < PA; u += 8) {
                    const float* row = P + (long long)wrapd(cu0 + u, H2) * V.rs;
                    const unsigned sb = smem_addr(pl + u * PAS);
                    for (int v = lane; v < PA; v += 32)
                        cp_async4s(sb + 4u * v, row + (inner ? cv0 + v : wrapd(cv0 + v, W2)));
                }
            } else {
                // transposed channel (rs = 1): walk along its memory rows, plane column v
                for (int v = warp; v < PA; v += 8) {
                    const float* col = P + (long long)wrapd(cv0 + v, W2) * V.cs;
                    for (int u = lane; u < PA; u += 32)
                        cp_async4s(smem_addr(pl + u * PAS + v), col + wrapd(cu0 + u, H2) * V.rs);
                }
            }
        }
    }
    cp_async_wait_all();
    __syncthreads();
    if (pp.first_odd) dfba_passes<NT, SYN, true>(planes, tmp, J.nst, pp);
    else dfba_passes<NT, SYN, false>(planes, tmp, J.nst, pp);
    // store the 64 x 64 tile: plane-local rows / columns [HALO/2, HALO/2 + 32)
    constexpr int T2 = DFBA_TILE / 2, H6 = HALO / 2;
    if (!SYN) {
        const int cub = y0 / 2, cvb = x0 / 2;
        for (int q = 0; q < 4; q++) {
            const View& V = J.comp[q];
            float* P = base_ptr(B, V.b) + V.off;
            const float* pl = planes + q * PL + H6 * PAS + H6;
            if (V.cs == 1) {
                // lane = plane column: each warp store is a run of one array row
                const int cv = cvb + lane;
                for (int u = warp; u < T2; u += 8) {
                    const int cu = cub + u;
                    if (cu < H2 && cv < W2) P[(long long)cu * V.rs + cv] = pl[u * PAS + lane];
                }
            } else {
                // transposed: lane = plane row, a run along the array's contiguous axis
                const int cu = cub + lane;
                for (int v = warp; v < T2; v += 8) {
                    const int cv = cvb + v;
                    if (cu < H2 && cv < W2) P[(long long)cu * V.rs + (long long)cv * V.cs] = pl[lane * PAS + v];
                }
            }
        }
    } else {
        float* Do = base_ptr(B, J.D.b) + J.D.off;
        static_assert(HALO % 2 == 0 && DFBA_TILE % 2 == 0, "column pairs start on even plane columns");
        if ((reinterpret_cast<uintptr_t>(Do) & 7) == 0 && (J.D.rs & 1) == 0) {
            // image row r per warp step, lane k = column pair (2k, 2k + 1): plane column
            // HALO/2 + k of the two planes of row parity (HALO + r) & 1, one 8-byte store
            const int x = x0 + 2 * lane;
            for (int r = warp; r < DFBA_TILE; r += 8) {
                const int y = y0 + r;
                if (y >= H) break;
                const int rr = HALO + r;
                const float* p = planes + 2 * (rr & 1) * PL + (rr >> 1) * PAS + H6 + lane;
                float* dst = Do + (long long)y * J.D.rs + x;
                if (x + 1 < W) *reinterpret_cast<float2*>(dst) = make_float2(p[0], p[PL]);
                else if (x < W) dst[0] = p[0];
            }
        } else {
            for (int k = threadIdx.x; k < DFBA_TILE * DFBA_TILE; k += blockDim.x) {
                int r = k / DFBA_TILE, c = k - r * DFBA_TILE;
                int y = y0 + r, x = x0 + c;
                if (y < H && x < W) {
                    int rr = HALO + r, cc = HALO + c;
                    Do[(long long)y * J.D.rs + x] = planes[(2 * (rr & 1) + (cc & 1)) * PL + (rr >> 1) * PAS + (cc >> 1)];
                }
            }
        }
    }
}

// ============================================================ k_dfb_b
// Tile frame for an NT-tap prototype (reach R = NT - 1 per pass): RB = 16 + 2R
// rows (R-row halo) by CB = 128 staged columns, rows stored with stride CBS.
// Shared-memory column x of tile row r holds column c0 + x - r - i*q of the
// row's coset array (q the parent row, c0 the tile's first output column):
//   - the shear by i*q turns the slope-i stencil (row offset a, column offset
//     -i*a + (b-a)/2) into one NT x NT pattern for every i, a parallelogram
//     that steps one column left per row;
//   - the extra column per row straightens it: target (r, x) reads the
//     rectangle rows [r + DB, r + DB + NT), columns [x + DB, x + DB + NT).
// So a pass is a separable NT x NT stencil on a plain grid.  COLS outputs per
// row (an R-column halo on each side; a multiple of 4); the output rows of a
// tile are shifted one column per row, which still cuts every array row into
// whole tiles because the arrays are periodic along their rows.
// The two coset arrays start MARGIN floats into their buffers; the pass-1
// source array is shifted by D more floats, so that every quad of targets and
// every source window of both passes starts on (or one float past) a 16-byte
// boundary.
template <int NT>
struct BGeo {
    static constexpr int R = NT - 1;
    static constexpr int CB = 128, CBS = CB + 4;
    static constexpr int COLS = (CB - 2 * R) & ~3;       // 120, 116, 112
    static constexpr int RB = DFBB_ROWS + 2 * R;
    static constexpr int MARGIN = 8;                    // reads of unused quads stay inside the buffer
    static constexpr int SMB = RB * CBS + 2 * MARGIN;   // floats per tile array
    static constexpr int D = NT == 4 ? 2 : 0;
};
static_assert(BGeo<4>::COLS == DFBB_COLS && dfbb_cols(4) == BGeo<4>::COLS && dfbb_cols(6) == BGeo<6>::COLS &&
                  dfbb_cols(8) == BGeo<8>::COLS,
              "host and device tile widths");
static_assert(2 * BGeo<8>::SMB * 4 <= 48 * 1024, "static shared memory");

// The passes of a stage with the first target coset odd (FO) or even.  Pass 1
// updates the first target coset F from the other one, S, over the rows and
// columns pass 2 reads; pass 2 updates S on the output tile.  A pass targets
// quads of 4 columns starting at X (16-byte aligned in its target array);
// the window of a quad, columns [x + DB, x + DB + NT + 3) of a source row,
// starts M floats past a 16-byte boundary.
template <int NT, bool FO>
struct BPass {
    using G = BGeo<NT>;
    static constexpr int R = G::R;
    static constexpr int DB1 = FO ? -(NT - 2) / 2 : -NT / 2;
    static constexpr int DB2 = FO ? -NT / 2 : -(NT - 2) / 2;
    // pass 1: F rows [R + DB2, R + DB2 + ROWS + R), columns [R + DB2, 2R + DB2 + COLS)
    static constexpr int R10 = R + DB2, R11 = R + DB2 + DFBB_ROWS + R;
    static constexpr int X1 = (R + DB2) & ~3;
    static constexpr int NQ1 = (2 * R + DB2 + G::COLS - X1 + 3) / 4;
    static constexpr int M1 = ((G::D + X1 + DB1) % 4 + 4) % 4;
    // pass 2: S rows [R, R + ROWS), columns [R, R + COLS)
    static constexpr int X2 = R - (R + G::D) % 4;
    static constexpr int NQ2 = (R + G::COLS - X2 + 3) / 4;
    static constexpr int M2 = ((X2 + DB2) % 4 + 4) % 4;
    static_assert(R10 + DB1 >= 0 && R11 - 1 + DB1 + NT - 1 < G::RB, "pass-1 rows inside the tile");
    static_assert(R + DB2 >= R10 && R + DFBB_ROWS - 1 + DB2 + NT - 1 < R11, "pass 2 reads pass-1 rows");
    static_assert(NQ1 <= 32 && NQ2 <= 32, "one quad per lane");
    static_assert(X1 + DB1 - M1 >= -G::MARGIN && X2 + DB2 - M2 >= -G::MARGIN, "left windows inside the margin");
    // right edge: the last quad's window, read as whole 16-byte chunks, ends inside the margin
    static constexpr int NCH1 = (M1 + NT + 6) / 4, NCH2 = (M2 + NT + 6) / 4;
    static_assert(X1 + 4 * NQ1 - 4 + DB1 - M1 + 4 * NCH1 <= G::CBS + G::MARGIN - G::D &&
                      X2 + 4 * NQ2 - 4 + DB2 - M2 + 4 * NCH2 <= G::CBS + G::MARGIN - G::D,
                  "right windows inside the margin");
    static_assert(X1 + 4 * NQ1 <= G::CBS && X2 + 4 * NQ2 + G::D <= G::CBS, "target quads inside their rows");
};

// The NT + 3 samples of a quad's window in one source row: p is 16-byte
// aligned, the window starts at p[M]
template <int NT, int M>
struct QWin {
    static constexpr int NCH = (M + NT + 3 + 3) / 4;
    float v[4 * NCH];
    __device__ __forceinline__ void load(const float* p) {
#pragma unroll
        for (int k = 0; k < NCH; k++) {
            const float4 t = reinterpret_cast<const float4*>(p)[k];
            v[4 * k] = t.x;
            v[4 * k + 1] = t.y;
            v[4 * k + 2] = t.z;
            v[4 * k + 3] = t.w;
        }
    }
};

__device__ __forceinline__ float2 f2(float a, float b) { return make_float2(a, b); }

// the row sums h(x + j) = sum_b bt[b] S[x + j + DB + b], j < 4, of one window, in b
// order; columns j and j + 1 in one paired instruction where the pair sits in
// adjacent loaded registers
template <int NT, int M>
__device__ __forceinline__ void quad_rowsums(const QWin<NT, M>& w, float2& h01, float2& h23) {
    constexpr float b0 = fan_tap(NT, 0);
    h01 = __fmul2_rn(f2(b0, b0), f2(w.v[M], w.v[M + 1]));
    h23 = __fmul2_rn(f2(b0, b0), f2(w.v[M + 2], w.v[M + 3]));
#pragma unroll
    for (int b = 1; b < NT; b++) {
        const float bt = fan_tap(NT, b);
        h01 = __ffma2_rn(f2(bt, bt), f2(w.v[M + b], w.v[M + b + 1]), h01);
        h23 = __ffma2_rn(f2(bt, bt), f2(w.v[M + b + 2], w.v[M + b + 3]), h23);
    }
}

// One ladder pass: for every target quad T[r][x .. x+3] of rows [R0, R1),
//   T[r][x+j] = alpha T[r][x+j] + gamma sum_ia bt[ia] h(r + DB + ia, x + j),
//   h(rho, c) = sum_b bt[b] S[rho][c + DB + b].
// Lane k takes the quad at column X + 4k (k < NQ); warp w walks the rows
// [R0 + w KC, R0 + (w+1) KC) down its quad with the NT row sums of the current
// target in registers, forming one new row sum per target.  Every sum is
// accumulated in the order of the scalar definition (taps in index order, the
// first a product), so each element rounds as a plain loop would round it.
template <int NT, int R0, int R1, int X, int NQ, int DB, int M, int TH>
__device__ __forceinline__ void ladder_quads(float* T, const float* S, float alpha, float gamma) {
    constexpr int CBS = BGeo<NT>::CBS, NWARPS = TH / 32;
    constexpr int NR = R1 - R0, KC = (NR + NWARPS - 1) / NWARPS;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int r0 = R0 + warp * KC;
    if (lane >= NQ || warp >= NWARPS || r0 >= R1) return;
    const int x = X + 4 * lane;
    const float* s = S + (r0 + DB) * CBS + (x + DB - M);
    float* t = T + r0 * CBS + x;
    const float2 al = f2(alpha, alpha), ga = f2(gamma, gamma);
    float2 g01[NT], g23[NT];    // row sums of source rows r + DB + ia of the current target row r
#pragma unroll
    for (int ia = 0; ia < NT - 1; ia++) {
        QWin<NT, M> w;
        w.load(s + ia * CBS);
        quad_rowsums<NT, M>(w, g01[ia], g23[ia]);
    }
    // a loop unrolled twice at most: the whole pass stays a few hundred instructions,
    // so the blocks of an SM in their different phases share the instruction cache
    const int steps = min(KC, R1 - r0);
    s += (NT - 1) * CBS;
#pragma unroll 2
    for (int k = 0; k < steps; k++, s += CBS, t += CBS) {
        {
            QWin<NT, M> w;
            w.load(s);
            quad_rowsums<NT, M>(w, g01[NT - 1], g23[NT - 1]);
        }
        constexpr float b0 = fan_tap(NT, 0);
        float2 a01 = __fmul2_rn(f2(b0, b0), g01[0]);
        float2 a23 = __fmul2_rn(f2(b0, b0), g23[0]);
#pragma unroll
        for (int ia = 1; ia < NT; ia++) {
            const float bt = fan_tap(NT, ia);
            a01 = __ffma2_rn(f2(bt, bt), g01[ia], a01);
            a23 = __ffma2_rn(f2(bt, bt), g23[ia], a23);
        }
        float4* tp = reinterpret_cast<float4*>(t);
        const float4 tv = *tp;
        const float2 o01 = __ffma2_rn(al, f2(tv.x, tv.y), __fmul2_rn(ga, a01));
        const float2 o23 = __ffma2_rn(al, f2(tv.z, tv.w), __fmul2_rn(ga, a23));
        *tp = make_float4(o01.x, o01.y, o23.x, o23.y);
#pragma unroll
        for (int ia = 0; ia < NT - 1; ia++) {
            g01[ia] = g01[ia + 1];
            g23[ia] = g23[ia + 1];
        }
    }
}

template <int CB>
__device__ __forceinline__ int wrap_fast(int v, int C) {
    // v in [0, C + CB): one subtraction when C >= CB, a remainder otherwise
    return v < C ? v : (C >= CB ? v - C : v % C);
}

template <int NT, bool FO, int TH>
__device__ __forceinline__ void dfb_b_passes(float* F, float* Sx, const PassParams& pp) {
    using P = BPass<NT, FO>;
    constexpr int R = BGeo<NT>::R;
    ladder_quads<NT, P::R10, P::R11, P::X1, P::NQ1, P::DB1, P::M1, TH>(F, Sx, pp.a1, pp.g1);
    __syncthreads();
    ladder_quads<NT, R, R + DFBB_ROWS, P::X2, P::NQ2, P::DB2, P::M2, TH>(Sx, F, pp.a2, pp.g2);
}

// One tile of a row-split stage (sE, sO: BGeo<NT>::SMB floats of shared memory
// each, 16-byte aligned), first target coset odd (FO = pp.first_odd) or even;
// RESIDENT: the channel arrays may live in shared memory (the tail kernel).
// The first TH threads of the block (a multiple of 128) do the work; every
// thread of the block must call it (it holds barriers).
template <bool SYN, int NT, bool FO, bool RESIDENT, int TH>
__device__ __forceinline__ void dfb_b_tile(const DfbBJob& J, int tile, const Bases& B, const PassParams& pp,
                                           float* sE, float* sO) {
    using G = BGeo<NT>;
    constexpr int R = G::R, RB = G::RB, CB = G::CB, CBS = G::CBS, COLS = G::COLS;
    const int ty = tile / J.tiles_x, tx = tile - ty * J.tiles_x;
    const int t0 = ty * DFBB_ROWS, c0 = tx * COLS;
    const int R2 = J.R2, C = J.C, i = J.i;
    static_assert(TH % 128 == 0 && TH <= 256, "four or eight working warps");
    constexpr int NW = TH / 32;   // working warps
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const bool worker = threadIdx.x < TH;
    constexpr bool fo = FO;
    // the first target coset's array at the margin, the other D floats further
    float* const arrE = sE + G::MARGIN + (fo ? G::D : 0);
    float* const arrO = sO + G::MARGIN + (fo ? 0 : G::D);
    // inputs: analysis reads the parent's cosets, synthesis the children.
    // Smem row r <-> coset row t0 - R + r; smem column x <-> array column
    // (c0 + x - r - i*q) mod C for parent row q = 2*(t0 - R + r) + parity
    const View V0 = SYN ? J.c0 : J.pe, V1 = SYN ? J.c1 : J.po;
    const float* const P0 = base_ptr(B, V0.b) + V0.off;
    const float* const P1 = base_ptr(B, V1.b) + V1.off;
    if (!worker) {
    } else if ((!RESIDENT || (!__isShared(P0) && !__isShared(P1))) && V0.cs == 1 && V1.cs == 1) {
        // row-major arrays.  Warp w stages rows w, w + NW, ... of both parities; lane
        // 2k + p first places row w + NW k of parity p (array row and start column, one
        // modular reduction for all of them), then the warp copies the rows one by one,
        // taking each row's placement from its lane.
        constexpr int RPW = (RB + NW - 1) / NW;
        static_assert(2 * RPW <= 32, "one lane per (row, parity) of a warp");
        const int lp = lane & 1, rl0 = warp + NW * (lane >> 1), tl = t0 - R + rl0;
        const int vl = wrapd(c0 - rl0 - i * (2 * tl + lp), C);
        const int ul = wrapd(tl, R2);
        const long long rs0 = V0.rs, rs1 = V1.rs;
#pragma unroll 1
        for (int kk = 0; kk < RPW; kk++) {
            const int r = warp + NW * kk;
            if (r >= RB) break;
#pragma unroll
            for (int par = 0; par < 2; par++) {
                const int u = __shfl_sync(0xffffffffu, ul, 2 * kk + par);
                const int vs = __shfl_sync(0xffffffffu, vl, 2 * kk + par);
                const float* row = par ? P1 + u * rs1 : P0 + u * rs0;
                const unsigned sb = smem_addr((par ? arrO : arrE) + r * CBS);
                if (vs + CB <= C) {                  // the window does not wrap: no per-element checks
                    const float* src = row + vs;
#pragma unroll
                    for (int x = lane; x < CB; x += 32) cp_async4s(sb + 4u * x, src + x);
                } else {
#pragma unroll
                    for (int x = lane; x < CB; x += 32) cp_async4s(sb + 4u * x, row + wrap_fast<CB>(vs + x, C));
                }
            }
        }
    } else {
        for (int par = 0; par < 2; par++) {
            const View V = par ? V1 : V0;
            const float* P = par ? P1 : P0;
            float* S = par ? arrO : arrE;
            if (RESIDENT && __isShared(P)) {
                // a tail kernel's resident channel array: plain copies of the sheared rows
                for (int r = warp; r < RB; r += NW) {
                    const int tu = t0 - R + r;
                    const float* row = P + (long long)wrapd(tu, R2) * V.rs;
                    const int vs = c0 - r - i * (2 * tu + par);
                    for (int x = lane; x < CB; x += 32) S[r * CBS + x] = row[(long long)wrapd(vs + x, C) * V.cs];
                }
            } else if (V.cs == 1) {
                for (int r = warp; r < RB; r += NW) {
                    const int tu = t0 - R + r;
                    const float* row = P + (long long)wrapd(tu, R2) * V.rs;
                    const int vs = wrapd(c0 - r - i * (2 * tu + par), C);
                    const unsigned sb = smem_addr(S + r * CBS);
                    for (int x = lane; x < CB; x += 32) cp_async4s(sb + 4u * x, row + wrap_fast<CB>(vs + x, C));
                }
            } else {
                // transposed array (contiguous along the rows t): lane r < RB takes smem row
                // r, and at step j tile column x = (j + (2i + 1) r) mod CB, whose array column
                // (c0 - r - i (2 tu + par) + x) mod C is the same for all rows until x wraps,
                // so a warp reads a run of consecutive t
                static_assert(RB <= 32 && (CB & (CB - 1)) == 0, "one lane per tile row; CB a power of two");
                const int tu = t0 - R + lane;
                const int vr = wrapd(c0 - lane - i * (2 * tu + par), C);
                const int sh = ((2 * i + 1) * lane) & (CB - 1);
                const float* rowp = P + (long long)wrapd(tu, R2) * V.rs;
                const unsigned sb = smem_addr(S + lane * CBS);
                if (lane < RB) {
                    for (int j = warp; j < CB; j += NW) {
                        const int x = (j + sh) & (CB - 1);
                        cp_async4s(sb + 4u * x, rowp + (long long)wrap_fast<CB>(vr + x, C) * V.cs);
                    }
                }
            }
        }
    }
    cp_async_wait_all();
    __syncthreads();
    if (FO) dfb_b_passes<NT, true, TH>(arrO, arrE, pp);
    else dfb_b_passes<NT, false, TH>(arrE, arrO, pp);
    __syncthreads();
    if (!worker) return;
    // outputs: analysis writes the children, synthesis the parent's cosets.  Output
    // (rr, u) of the tile is smem (R + rr, R + u), array column c0 + u - rr - i (2t + par)
    const int ncol = min(COLS, C - c0);
    const View W0 = SYN ? J.pe : J.c0, W1 = SYN ? J.po : J.c1;
    float* const Q0 = base_ptr(B, W0.b) + W0.off;
    float* const Q1 = base_ptr(B, W1.b) + W1.off;
    if (W0.cs == 1 && W1.cs == 1) {
        // row-major arrays: warp w writes rows w, w + NW, ... of both parities, placed by
        // its lanes as in the row-major staging
        constexpr int RPW = DFBB_ROWS / NW;
        static_assert(DFBB_ROWS % NW == 0 && 2 * RPW <= 32, "one lane per (row, parity) of a warp");
        const int lp = lane & 1, rl = warp + NW * (lane >> 1), tl = t0 + rl;
        const int vl = wrapd(c0 - rl - i * (2 * tl + lp), C);
        const long long rs0 = W0.rs, rs1 = W1.rs;
#pragma unroll 1
        for (int kk = 0; kk < RPW; kk++) {
            const int rr = warp + NW * kk, t = t0 + rr;
            if (t >= R2) break;
#pragma unroll
            for (int par = 0; par < 2; par++) {
                const int vs = __shfl_sync(0xffffffffu, vl, 2 * kk + par);
                float* row = par ? Q1 + t * rs1 : Q0 + t * rs0;
                const float* srow = (par ? arrO : arrE) + (R + rr) * CBS + R;
                if (vs + ncol <= C) {
                    float* dst = row + vs;
#pragma unroll
                    for (int xx = lane; xx < COLS; xx += 32)
                        if (xx < ncol) dst[xx] = srow[xx];
                } else {
#pragma unroll
                    for (int xx = lane; xx < COLS; xx += 32)
                        if (xx < ncol) row[wrap_fast<CB>(vs + xx, C)] = srow[xx];
                }
            }
        }
    } else {
        for (int par = 0; par < 2; par++) {
            const View V = par ? W1 : W0;
            float* P = par ? Q1 : Q0;
            const float* S = par ? arrO : arrE;
            if (V.cs == 1) {
                for (int rr = warp; rr < DFBB_ROWS; rr += NW) {
                    const int t = t0 + rr;
                    if (t >= R2) break;
                    float* row = P + (long long)t * V.rs;
                    const int vs = wrapd(c0 - rr - i * (2 * t + par), C);
                    const float* srow = S + (R + rr) * CBS + R;
                    for (int xx = lane; xx < ncol; xx += 32) row[wrap_fast<CB>(vs + xx, C)] = srow[xx];
                }
            } else {
                // transposed subband (contiguous along t): lanes 0..15 take the tile rows of
                // one column chunk j, lanes 16..31 those of chunk j + 1; row rr writes tile
                // column xx = (j + (2i + 1) rr) mod COLS, whose subband column
                // (c0 - rr - i (2 t + par) + xx) mod C is the same for all rows until xx wraps
                static_assert(DFBB_ROWS == 16, "half a warp per column chunk");
                const int rr = lane & 15, t = t0 + rr;
                const int vr = wrapd(c0 - rr - i * (2 * t + par), C);
                const int sh = wrapd((2 * i + 1) * rr, COLS);
                float* colp = P + (long long)t * V.rs;
                const float* srow = S + (R + rr) * CBS + R;
                if (t < R2) {
                    for (int j = 2 * warp + (lane >> 4); j < COLS; j += 2 * NW) {
                        int xx = j + sh;
                        xx -= xx >= COLS ? COLS : 0;
                        if (xx < ncol) colp[(long long)wrap_fast<COLS>(vr + xx, C) * V.cs] = srow[xx];
                    }
                }
            }
        }
    }
}

}  // namespace cvc
