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

__constant__ float c_bt[4] = {-1.f / 16, -9.f / 16, 9.f / 16, 1.f / 16};

// ============================================================ k_dfb_a
constexpr int SA = DFBA_TILE + 2 * DFBA_HALO;  // 88: tile + halo, image samples
constexpr int PA = SA / 2;                     // 44: polyphase plane side
constexpr int PAS = PA + 1;                    // padded plane row stride

// tap t = 4*ia + ib, a = 2ia-3, b = 2ib-3; image offset of the tap for a
// target of class (pr, pc) at stage 1 / 2
__host__ __device__ constexpr int tap_dy(int stage, int pr, int pc, int t) {
    return stage == 1 ? ((2 * (t >> 2) - 3) + (2 * (t & 3) - 3)) / 2
                      : (pr == pc ? (2 * (t >> 2) - 3) : (2 * (t & 3) - 3));
}
__host__ __device__ constexpr int tap_dx(int stage, int pr, int pc, int t) {
    return stage == 1 ? ((2 * (t >> 2) - 3) - (2 * (t & 3) - 3)) / 2
                      : (pr == pc ? (2 * (t & 3) - 3) : (2 * (t >> 2) - 3));
}
__host__ __device__ constexpr int fdiv2(int a) { return a >= 0 ? a / 2 : -((1 - a) / 2); }

// one pass over target class (PR, PC): plane rows / columns [u0, u1) x [v0, v1)
template <int STAGE, int PR, int PC>
__device__ __forceinline__ void dfba_class_pass(float* planes, int n, float alpha, float gamma) {
    const int lo = 3 * n, hi = SA - 3 * n;
    const int u0 = (lo - PR + 1) / 2, u1 = (hi - 1 - PR) / 2 + 1;
    const int v0 = (lo - PC + 1) / 2, v1 = (hi - 1 - PC) / 2 + 1;
    const int nu = u1 - u0, nv = v1 - v0;
    float* T = planes + (2 * PR + PC) * PA * PAS;
    for (int k = threadIdx.x; k < nu * nv; k += blockDim.x) {
        const int u = u0 + k / nv, v = v0 + k % nv;
        float acc = 0.f;
#pragma unroll
        for (int t = 0; t < 16; t++) {
            const int dy = tap_dy(STAGE, PR, PC, t), dx = tap_dx(STAGE, PR, PC, t);
            const int sr = PR + dy, sc = PC + dx;
            const int q = ((sr & 1) << 1) | (sc & 1);
            const float* S = planes + q * PA * PAS;
            acc = fmaf(c_bt[t >> 2] * c_bt[t & 3], S[(u + fdiv2(sr)) * PAS + v + fdiv2(sc)], acc);
        }
        T[u * PAS + v] = fmaf(alpha, T[u * PAS + v], gamma * acc);
    }
}

template <int STAGE>
__device__ __forceinline__ void dfba_pass(float* planes, int n, int odd, float alpha, float gamma) {
    if (STAGE == 1) {
        // stage 1: odd coset = classes 01, 10; even = 00, 11
        if (odd) { dfba_class_pass<1, 0, 1>(planes, n, alpha, gamma); dfba_class_pass<1, 1, 0>(planes, n, alpha, gamma); }
        else { dfba_class_pass<1, 0, 0>(planes, n, alpha, gamma); dfba_class_pass<1, 1, 1>(planes, n, alpha, gamma); }
    } else {
        // stage 2: odd coset = classes 11 (family c), 01 (family r); even = 00 (c), 10 (r)
        if (odd) { dfba_class_pass<2, 1, 1>(planes, n, alpha, gamma); dfba_class_pass<2, 0, 1>(planes, n, alpha, gamma); }
        else { dfba_class_pass<2, 0, 0>(planes, n, alpha, gamma); dfba_class_pass<2, 1, 0>(planes, n, alpha, gamma); }
    }
    __syncthreads();
}

template <bool SYN>
__global__ void __launch_bounds__(256) k_dfb_a(const DfbAJob* __restrict__ jobs, const int* __restrict__ block_job,
                                               Bases B, PassParams pp) {
    __shared__ float planes[4 * PA * PAS];
    const DfbAJob& J = jobs[block_job[blockIdx.x]];
    const int tile = blockIdx.x - J.first_block;
    const int ty = tile / J.tiles_x, tx = tile - ty * J.tiles_x;
    const int y0 = ty * DFBA_TILE, x0 = tx * DFBA_TILE;
    const int H = J.H, W = J.W, H2 = H / 2, W2 = W / 2;
    // plane-local (u, v) of class (pr, pc) <-> image (y0 - 12 + 2u + pr, x0 - 12 + 2v + pc);
    // class-array index ((y0 - 12)/2 + u, (x0 - 12)/2 + v), periodic in (H/2, W/2)
    const int cu0 = (y0 - DFBA_HALO) / 2, cv0 = (x0 - DFBA_HALO) / 2;
    if (!SYN) {
        const float* Dp = B.p[J.D.b] + J.D.off;
        for (int k = threadIdx.x; k < SA * SA; k += blockDim.x) {
            int r = k / SA, c = k - r * SA;
            int y = wrapd(y0 - DFBA_HALO + r, H), x = wrapd(x0 - DFBA_HALO + c, W);
            planes[(2 * (r & 1) + (c & 1)) * PA * PAS + (r >> 1) * PAS + (c >> 1)] = Dp[(long long)y * J.D.rs + x];
        }
    } else {
        for (int q = 0; q < 4; q++) {
            const View& V = J.comp[q];
            const float* P = B.p[V.b] + V.off;
            const bool trans = V.cs != 1;
            for (int k = threadIdx.x; k < PA * PA; k += blockDim.x) {
                int a = k / PA, b = k - a * PA;
                int u = trans ? b : a, v = trans ? a : b;
                int cu = wrapd(cu0 + u, H2), cv = wrapd(cv0 + v, W2);
                planes[q * PA * PAS + u * PAS + v] = P[(long long)cu * V.rs + (long long)cv * V.cs];
            }
        }
    }
    __syncthreads();
    // analysis runs stage 1 then 2, synthesis stage 2 then 1
    if (!SYN) {
        dfba_pass<1>(planes, 1, pp.first_odd, pp.a1, pp.g1);
        dfba_pass<1>(planes, 2, !pp.first_odd, pp.a2, pp.g2);
        if (J.nst == 2) {
            dfba_pass<2>(planes, 3, pp.first_odd, pp.a1, pp.g1);
            dfba_pass<2>(planes, 4, !pp.first_odd, pp.a2, pp.g2);
        }
    } else {
        int n = 1;
        if (J.nst == 2) {
            dfba_pass<2>(planes, n++, pp.first_odd, pp.a1, pp.g1);
            dfba_pass<2>(planes, n++, !pp.first_odd, pp.a2, pp.g2);
        }
        dfba_pass<1>(planes, n++, pp.first_odd, pp.a1, pp.g1);
        dfba_pass<1>(planes, n++, !pp.first_odd, pp.a2, pp.g2);
    }
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
constexpr int RB = DFBB_ROWS + 6, CB = DFBB_COLS + 12;

// separable 4 x 4 pass in the sheared frame: target rows [r0, r1) x cols [x0, x1)
// of array T, sources in array S (rows r + (a + dr)/2 with dr = +1 for odd
// targets, -1 for even ones; columns x + (b - a)/2).
__device__ __forceinline__ void dfbb_pass(float* T, const float* S, float* Hs, int r0, int r1, int x0, int x1,
                                          int odd_target, float alpha, float gamma) {
    const int sr0 = r0 + (odd_target ? -1 : -2), sr1 = r1 + (odd_target ? 2 : 1);
    const int hx0 = x0 - 3, hw = x1 - hx0;
    // row sums h[rr][x'] = sum_b betat[b] * S[rr][x' + (b+3)/2]
    for (int k = threadIdx.x; k < (sr1 - sr0) * hw; k += blockDim.x) {
        const int rr = sr0 + k / hw, xx = hx0 + k % hw;
        const float* src = S + rr * CB + xx;
        float acc = c_bt[0] * src[0];
        acc = fmaf(c_bt[1], src[1], acc);
        acc = fmaf(c_bt[2], src[2], acc);
        Hs[rr * CB + xx] = fmaf(c_bt[3], src[3], acc);
    }
    __syncthreads();
    const int w = x1 - x0;
    // tap a (ia = 0..3, a = 2ia - 3): row r + (a + (odd ? 1 : -1))/2 = rb + ia, column x - (a+3)/2 = x - ia
    const int db = odd_target ? -1 : -2;
    for (int k = threadIdx.x; k < (r1 - r0) * w; k += blockDim.x) {
        const int r = r0 + k / w, x = x0 + k % w;
        const float* h = Hs + (r + db) * CB + x;
        float acc = c_bt[0] * h[0];
        acc = fmaf(c_bt[1], h[CB - 1], acc);
        acc = fmaf(c_bt[2], h[2 * CB - 2], acc);
        acc = fmaf(c_bt[3], h[3 * CB - 3], acc);
        float* t = T + r * CB + x;
        *t = fmaf(alpha, *t, gamma * acc);
    }
    __syncthreads();
}

__device__ __forceinline__ int wrap_fast(int v, int C) {
    // v in [0, C + CB): one subtraction when C >= CB, a remainder otherwise
    return v < C ? v : (C >= CB ? v - C : v % C);
}

template <bool SYN>
__global__ void __launch_bounds__(256) k_dfb_b(const DfbBJob* __restrict__ jobs, const int* __restrict__ block_job,
                                               Bases B, PassParams pp) {
    __shared__ float sE[RB * CB];
    __shared__ float sO[RB * CB];
    __shared__ float sH[RB * CB];
    const DfbBJob& J = jobs[block_job[blockIdx.x]];
    const int tile = blockIdx.x - J.first_block;
    const int ty = tile / J.tiles_x, tx = tile - ty * J.tiles_x;
    const int t0 = ty * DFBB_ROWS, c0 = tx * DFBB_COLS;
    const int R2 = J.R2, C = J.C, i = J.i;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nwarp = blockDim.x >> 5;
    // inputs: analysis reads the parent's cosets, synthesis the children.
    // Smem row r <-> coset row t0 - 3 + r; smem column x <-> sheared column c0 - 6 + x,
    // i.e. array column (c0 - 6 + x - i*q) mod C for parent row q = 2*(t0 - 3 + r) + parity
    for (int par = 0; par < 2; par++) {
        const View V = par ? (SYN ? J.c1 : J.po) : (SYN ? J.c0 : J.pe);
        const float* P = B.p[V.b] + V.off;
        float* S = par ? sO : sE;
        if (V.cs == 1) {
            for (int r = warp; r < RB; r += nwarp) {
                const int tu = t0 - 3 + r;
                const float* row = P + (long long)wrapd(tu, R2) * V.rs;
                const int vs = wrapd(c0 - 6 - i * (2 * tu + par), C);
                for (int x = lane; x < CB; x += 32) S[r * CB + x] = row[wrap_fast(vs + x, C)];
            }
        } else {
            for (int k = threadIdx.x; k < RB * CB; k += blockDim.x) {
                const int x = k / RB, r = k - x * RB;
                const int tu = t0 - 3 + r;
                const int v = wrapd(c0 - 6 + x - i * (2 * tu + par), C);
                S[r * CB + x] = P[(long long)wrapd(tu, R2) * V.rs + (long long)v * V.cs];
            }
        }
    }
    __syncthreads();
    // pass 1 covers what pass 2 needs; pass 2 covers the tile [3, 3+ROWS) x [6, 6+COLS)
    const int fo = pp.first_odd;
    if (fo) dfbb_pass(sO, sE, sH, 1, DFBB_ROWS + 4, 3, DFBB_COLS + 9, 1, pp.a1, pp.g1);
    else dfbb_pass(sE, sO, sH, 2, DFBB_ROWS + 5, 3, DFBB_COLS + 9, 0, pp.a1, pp.g1);
    if (fo) dfbb_pass(sE, sO, sH, 3, DFBB_ROWS + 3, 6, DFBB_COLS + 6, 0, pp.a2, pp.g2);
    else dfbb_pass(sO, sE, sH, 3, DFBB_ROWS + 3, 6, DFBB_COLS + 6, 1, pp.a2, pp.g2);
    // outputs: analysis writes the children, synthesis the parent's cosets
    const int ncol = min(DFBB_COLS, C - c0);
    for (int par = 0; par < 2; par++) {
        const View V = par ? (SYN ? J.po : J.c1) : (SYN ? J.pe : J.c0);
        float* P = B.p[V.b] + V.off;
        const float* S = par ? sO : sE;
        if (V.cs == 1) {
            for (int rr = warp; rr < DFBB_ROWS; rr += nwarp) {
                const int t = t0 + rr;
                if (t >= R2) break;
                float* row = P + (long long)t * V.rs;
                const int vs = wrapd(c0 - i * (2 * t + par), C);
                for (int xx = lane; xx < ncol; xx += 32) row[wrap_fast(vs + xx, C)] = S[(3 + rr) * CB + 6 + xx];
            }
        } else {
            for (int k = threadIdx.x; k < DFBB_ROWS * DFBB_COLS; k += blockDim.x) {
                const int xx = k / DFBB_ROWS, rr = k - xx * DFBB_ROWS;
                const int t = t0 + rr;
                if (t >= R2 || xx >= ncol) continue;
                const int v = wrapd(c0 + xx - i * (2 * t + par), C);
                P[(long long)t * V.rs + (long long)v * V.cs] = S[(3 + rr) * CB + 6 + xx];
            }
        }
    }
}

// ============================================================ launches
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
    } else {
        const DfbBJob* j = static_cast<const DfbBJob*>(L.d_jobs);
        if (syn) k_dfb_b<true><<<L.nblocks, 256, 0, st>>>(j, L.d_block_job, bases, pp);
        else k_dfb_b<false><<<L.nblocks, 256, 0, st>>>(j, L.d_block_job, bases, pp);
    }
    return cudaGetLastError();
}

}  // namespace cvc
