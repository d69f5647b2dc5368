// k_codec.cu -- the codec's element-wise and row-wise stages, each launch
// covering every stream of a batch:
//   colour conversion + 4:2:0 + padding (§3.1), quantisation with lowpass
//   normalisation and thresholding (§3.4-§3.6), K/P differencing (§3.7),
//   run-length coding of rows (§3.8), their inverses, and device-wide scans.
// Blocks find their stream / plane through block maps built at creation, so
// no grid depends on per-call sizes; per-call arguments (buffers) come from
// device records refreshed by one copy per call, and the coder state (frame
// index, state parity, the decoder's expectations) lives on the device.
#include <algorithm>

#include "k_codec.cuh"

namespace cvc {

__device__ __forceinline__ int mirror_idx(int a, int n) { return a < n ? a : 2 * n - 1 - a; }

// ------------------------------------------------------- step begin / commit
// §3.7: frame i of a stream (counted from its last reset) is a K-frame iff
// i % key_interval == 0; a decoder accepts a P-frame only with the index
// following the last frame it decoded, and only at scales its state covers.
__global__ void k_step_begin(const SDesc* __restrict__ sd, SCall* __restrict__ sc, SCtl* __restrict__ ctl, int n) {
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= n) return;
    SCall& C = sc[s];
    SCtl& T = ctl[s];
    if (C.reset) {
        T.enc_frame = 0;
        T.dec_next = -1;
        T.dec_floor = 0;
    }
    C.ecur = T.ecur;
    C.dcur = T.dcur;
    if (C.enc_on) {
        C.enc_key = (T.enc_frame % sd[s].key_interval) == 0;
        C.enc_index = (uint32_t)T.enc_frame;
    }
    if (C.dec_on) {
        C.dec_expect = T.dec_next;
        C.dec_floor = T.dec_floor;
        if (C.in_len_dev && C.in_len >= 0) {
            const size_t len = *C.in_len_dev;
            if (len < (size_t)C.in_len) C.in_len = (long long)len;
        }
    }
}

// The outcome of one stream's call.  Encoder: OVERFLOW when a code left int16,
// CAPACITY when the frame does not fit out_cap (out_len is then the size it
// needs); decoder: STATE for a P-frame without its reference (or below the
// state's scale floor), CORRUPT for a malformed or mismatched stream.  A
// successful call advances the coder state: the encoder's frame index and
// state parity; the decoder's parity, expected index and scale floor (a
// K-frame sets the floor to its own dropped levels, a P-frame can only raise
// it).  A failed call leaves it as it was.
__global__ void k_step_commit(const SDesc* __restrict__ sd, const SCall* __restrict__ sc, SResult* __restrict__ rs,
                              SCtl* __restrict__ ctl, int n) {
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= n) return;
    const SDesc& D = sd[s];
    const SCall& C = sc[s];
    SResult& R = rs[s];
    SCtl& T = ctl[s];
    cvc_batch_result out;
    out.enc_status = CVC_OK;
    out.dec_status = CVC_OK;
    out.out_len = 0;
    out.frame_type = -1;
    out.dec_frame_type = -1;
    out.dec_frame_index = 0;
    if (C.enc_on) {
        const bool mc = !C.enc_key && D.mv_range > 0;
        const long long need = D.hdr_bytes + 2LL * R.enc_tokens + (mc ? D.mv_bytes : 0);
        out.out_len = (size_t)need;
        out.frame_type = C.enc_key ? 0 : (mc ? 2 : 1);
        if (R.enc_err & EF_OVERFLOW) out.enc_status = CVC_ERR_OVERFLOW;
        else if (need > C.out_cap || (R.enc_err & EF_CAPACITY)) out.enc_status = CVC_ERR_CAPACITY;
        if (out.enc_status == CVC_OK && !C.no_commit) {
            T.ecur = 1 - T.ecur;
            T.enc_frame += 1;
        }
    }
    if (C.dec_on) {
        if (R.dec_err & EF_STATE) out.dec_status = CVC_ERR_STATE;
        else if (R.dec_err & (EF_CORRUPT | EF_MISMATCH)) out.dec_status = CVC_ERR_CORRUPT;
        if (out.dec_status == CVC_OK) {
            out.dec_frame_type = (int)R.dec_type;
            out.dec_frame_index = R.dec_index;
            if (!C.no_commit) {
                const int drop = (int)R.dec_drop;
                T.dcur = 1 - T.dcur;
                T.dec_next = (long long)R.dec_index + 1;
                T.dec_floor = R.dec_type == 0 ? drop : max(T.dec_floor, drop);
            }
        }
    }
    R.res = out;
    const cvc_status first = out.enc_status != CVC_OK ? out.enc_status : out.dec_status;
    if (C.async && first != CVC_OK && T.first_err == CVC_OK) T.first_err = first;
    if (C.res_dev) *C.res_dev = out;
    if (C.enc_on) {
        if (C.out_len_dev) *C.out_len_dev = out.out_len;
        if (C.type_dev) *C.type_dev = out.frame_type;
        if (C.enc_status_dev) *C.enc_status_dev = out.enc_status;
    }
    if (C.dec_on && C.dec_status_dev) *C.dec_status_dev = out.dec_status;
}

// ------------------------------------------------------------- colour
// YCoCg-R lifting (integer form of Table 1): Co = R-B, t = B + (Co>>1),
// Cg = G - t, Y = t + (Cg>>1).  One block per padded output row: rows
// [0, Hp) are luma rows, rows [Hp, Hp + Hcp) chroma rows (each writes its Co
// and Cg row; 2x2 rounded mean, odd edges replicated); padding mirrors about
// the last row / column.  8-bit storage (§3.1, §3.6): Table I's
// real-valued form instead, each component rounded to a byte, chroma offset
// by +127 and clamped to [0, 255].
// v / 2^sh rounded half away from zero (sh >= 1)
__device__ __forceinline__ int div_pow2_round(int v, int sh) {
    const int r = (abs(v) + (1 << (sh - 1))) >> sh;
    return v < 0 ? -r : r;
}

// luma of one pixel: YCoCg-R, or (8-bit storage) Table I's Y = (R + 2G + B)/4 rounded
__device__ __forceinline__ int luma_of(int R, int G, int B, bool st8) {
    if (st8) return (R + 2 * G + B + 2) >> 2;
    const int co = R - B, t = B + (co >> 1), cg = G - t;
    return t + (cg >> 1);
}

__global__ void k_colour_fwd_b(const SDesc* __restrict__ sd, const SCall* __restrict__ sc,
                               const int* __restrict__ blk_stream, float* __restrict__ planes,
                               uint8_t* __restrict__ luma0, uint8_t* __restrict__ luma1) {
    const int s = blk_stream[blockIdx.x];
    const SCall& C = sc[s];
    if (!C.enc_on) return;
    const SDesc& D = sd[s];
    const ColourGeom g = D.cg;
    const bool st8 = D.qp.st8;
    const int row = blockIdx.x - D.blk_colour;
    const uint8_t* rgb = C.rgb_in;
    const long long pitch = C.pitch_in;
    float* Y = planes + D.plane_off;
    if (row < g.Hp) {
        const uint8_t* src = rgb + (long long)mirror_idx(row, g.H) * pitch;
        float* out = Y + (long long)row * g.Wp;
        // streams with motion also keep the padded luma as bytes (Y is in [0, 255]) for the search
        uint8_t* lum = D.mv_range ? (C.ecur ? luma0 : luma1) + D.luma_off + (long long)row * g.Wp : nullptr;
        // four pixels per thread: three word loads, one float4 store, where the row is aligned
        const bool vec = (((uintptr_t)src | (uintptr_t)out | (uintptr_t)(lum ? lum : src)) & 3) == 0 &&
                         ((uintptr_t)out & 15) == 0;
        for (int x0 = 4 * threadIdx.x; x0 < g.Wp; x0 += 4 * blockDim.x) {
            int yv[4];
            if (vec && x0 + 4 <= g.W) {
                const uint32_t* w = reinterpret_cast<const uint32_t*>(src + 3 * x0);
                const uint32_t w0 = w[0], w1 = w[1], w2 = w[2];
                const int px[12] = {(int)(w0 & 255), (int)((w0 >> 8) & 255), (int)((w0 >> 16) & 255), (int)(w0 >> 24),
                                    (int)(w1 & 255), (int)((w1 >> 8) & 255), (int)((w1 >> 16) & 255), (int)(w1 >> 24),
                                    (int)(w2 & 255), (int)((w2 >> 8) & 255), (int)((w2 >> 16) & 255), (int)(w2 >> 24)};
#pragma unroll
                for (int k = 0; k < 4; k++) yv[k] = luma_of(px[3 * k], px[3 * k + 1], px[3 * k + 2], st8);
            } else {
#pragma unroll
                for (int k = 0; k < 4; k++) {
                    const int x = min(x0 + k, g.Wp - 1);
                    const uint8_t* p = src + 3 * mirror_idx(x, g.W);
                    yv[k] = luma_of(p[0], p[1], p[2], st8);
                }
            }
            if (vec && x0 + 4 <= g.Wp) {
                *reinterpret_cast<float4*>(out + x0) = make_float4((float)yv[0], (float)yv[1], (float)yv[2], (float)yv[3]);
                if (lum)
                    *reinterpret_cast<uint32_t*>(lum + x0) =
                        (uint32_t)yv[0] | ((uint32_t)yv[1] << 8) | ((uint32_t)yv[2] << 16) | ((uint32_t)yv[3] << 24);
            } else {
                for (int k = 0; k < 4 && x0 + k < g.Wp; k++) {
                    out[x0 + k] = (float)yv[k];
                    if (lum) lum[x0 + k] = (uint8_t)yv[k];
                }
            }
        }
    } else {
        const int cy = row - g.Hp;
        const int sy = mirror_idx(cy, g.Hc);
        const uint8_t* r0 = rgb + (long long)(2 * sy) * pitch;
        const uint8_t* r1 = rgb + (long long)min(2 * sy + 1, g.H - 1) * pitch;
        float* oco = Y + (long long)g.Hp * g.Wp + (long long)cy * g.Wcp;
        float* ocg = oco + (long long)g.Hcp * g.Wcp;
        for (int cx = threadIdx.x; cx < g.Wcp; cx += blockDim.x) {
            const int sx = mirror_idx(cx, g.Wc);
            const int c0 = 3 * (2 * sx), c1 = 3 * min(2 * sx + 1, g.W - 1);
            int sco = 0, scg = 0;
            const uint8_t* q[4] = {r0 + c0, r0 + c1, r1 + c0, r1 + c1};
#pragma unroll
            for (int k = 0; k < 4; k++) {
                const int R = q[k][0], G = q[k][1], Bv = q[k][2];
                if (st8) {
                    // Table I: Co = (R - B)/2, Cg = (2G - R - B)/4, rounded, +127, clamped to a byte
                    sco += min(max(div_pow2_round(R - Bv, 1) + 127, 0), 255);
                    scg += min(max(div_pow2_round(2 * G - R - Bv, 2) + 127, 0), 255);
                } else {
                    const int co = R - Bv, t = Bv + (co >> 1);
                    sco += co;
                    scg += G - t;
                }
            }
            oco[cx] = (float)((sco + 2) >> 2);
            ocg[cx] = (float)((scg + 2) >> 2);
        }
    }
}

__device__ __forceinline__ int round_clamp(float v, int lo, int hi) {
    float r = roundf(v);
    r = fminf(fmaxf(r, (float)lo), (float)hi);
    return (int)r;
}

// Decoder end: normalise by the scale's DC gain, round (ties away from zero)
// and clamp the reconstructed planes, bilinear (9,3,3,1)/16 chroma
// upsampling with centred siting and clamped edges, inverse YCoCg-R (8-bit
// storage: Table I's inverse after removing the chroma offset), clamp to
// [0, 255].  One block per output row.  A stream whose bitstream was
// rejected leaves its output untouched.
__global__ void k_colour_inv_b(const ScaleDesc* __restrict__ sdesc, const SCall* __restrict__ sc,
                               const SResult* __restrict__ rs, const int* __restrict__ blk_stream,
                               const float* __restrict__ rplanes, const float* __restrict__ dcoef) {
    const int s = blk_stream[blockIdx.x];
    const SCall& C = sc[s];
    if (!C.dec_on || rs[s].dec_err) return;
    const ScaleDesc& D = sdesc[s];
    const float* base = D.src ? dcoef : rplanes;
    const float norm = D.norm;
    const int y = blockIdx.x - D.blk0;
    const float* Yrow = base + D.off[0] + (long long)y * D.rs_y;
    const float* Co = base + D.off[1];
    const float* Cg = base + D.off[2];
    const int Hc = D.Hc, Wc = D.Wc;
    const int i0 = min(y >> 1, Hc - 1), i1 = (y & 1) ? min((y >> 1) + 1, Hc - 1) : max((y >> 1) - 1, 0);
    const float* P[2][2] = {{Co + (long long)i0 * D.rs_c, Co + (long long)i1 * D.rs_c},
                            {Cg + (long long)i0 * D.rs_c, Cg + (long long)i1 * D.rs_c}};
    uint8_t* orow = C.rgb_out + (long long)y * C.pitch_out;
    const bool vec = ((uintptr_t)orow & 3) == 0;
    const bool st8 = D.st8;
    const int clo = st8 ? 0 : -255;    // chroma bytes (offset by 127), or YCoCg-R chroma
    // four pixels per thread: their chroma columns x/2 - 1 .. x/2 + 2 (clamped) are rounded once
    for (int x0 = 4 * threadIdx.x; x0 < D.W; x0 += 4 * blockDim.x) {
        const int jb = x0 >> 1;
        int cv[2][2][4];
#pragma unroll
        for (int k = 0; k < 4; k++) {
            const int j = min(max(jb - 1 + k, 0), Wc - 1);
#pragma unroll
            for (int q = 0; q < 2; q++)
#pragma unroll
                for (int r = 0; r < 2; r++) cv[q][r][k] = round_clamp(P[q][r][j] * norm, clo, 255);
        }
        uint32_t px[3] = {0, 0, 0};
#pragma unroll
        for (int k = 0; k < 4; k++) {
            const int x = x0 + k;
            if (x >= D.W) break;
            const int yy = round_clamp(Yrow[x] * norm, 0, 255);
            // columns min(x/2, Wc-1) and, for odd x, min(x/2 + 1, Wc-1), for even x, x/2 - 1 (>= 0)
            const int i0 = (k >> 1) + 1, i1 = (k & 1) ? (k >> 1) + 2 : (k >> 1);
            int c[2];
#pragma unroll
            for (int q = 0; q < 2; q++)
                c[q] = (9 * cv[q][0][i0] + 3 * cv[q][1][i0] + 3 * cv[q][0][i1] + cv[q][1][i1] + 8) >> 4;
            int R, G, Bv;
            if (st8) {                   // Table I inverse: R = Y + Co - Cg, G = Y + Cg, B = Y - Co - Cg
                const int co = c[0] - 127, cg = c[1] - 127;
                R = yy + co - cg;
                G = yy + cg;
                Bv = yy - co - cg;
            } else {
                const int t = yy - (c[1] >> 1);
                G = c[1] + t;
                Bv = t - (c[0] >> 1);
                R = Bv + c[0];
            }
            const uint32_t rgb3[3] = {(uint32_t)min(max(R, 0), 255), (uint32_t)min(max(G, 0), 255),
                                      (uint32_t)min(max(Bv, 0), 255)};
#pragma unroll
            for (int b = 0; b < 3; b++) px[(3 * k + b) >> 2] |= rgb3[b] << (8 * ((3 * k + b) & 3));
        }
        if (vec && x0 + 4 <= D.W) {
            uint32_t* o = reinterpret_cast<uint32_t*>(orow + 3 * x0);
            o[0] = px[0];
            o[1] = px[1];
            o[2] = px[2];
        } else {
            for (int b = 0; b < 12 && x0 + b / 3 < D.W; b++) orow[3 * x0 + b] = (uint8_t)(px[b >> 2] >> (8 * (b & 3)));
        }
    }
}

// ------------------------------------------------------ quantisation + K/P
__device__ __forceinline__ int quant(float c, bool low, const QuantParams& q, uint32_t* err) {
    float t;
    if (low) t = c * q.low_scale;                    // exact power-of-two normalisation
    else t = (fabsf(c) >= q.threshold) ? c : 0.0f;
    float v = roundf(t / (low ? q.qpl : q.qph));     // IEEE division, ties away from zero
    // 8-bit storage (§3.6): the rounded code is kept in a byte
    if (q.st8) v = low ? fminf(fmaxf(v, 0.0f), 255.0f) : fminf(fmaxf(v, -128.0f), 127.0f);
    if (!(fabsf(v) <= 32767.0f)) {
        atomicOr(err, EF_OVERFLOW);
        return 0;
    }
    return (int)v;
}

// codes q (the next coder state) and residuals r of one frame per stream;
// a block covers ELEM_BLOCK elements of one plane, ELEM_PER_THREAD per thread
__global__ void __launch_bounds__(ELEM_THREADS) k_quant_b(const float* __restrict__ coef, int16_t* est0,
                                                          int16_t* est1, const PDesc* __restrict__ pd,
                                                          const int* __restrict__ blk_plane,
                                                          const SDesc* __restrict__ sd, const SCall* __restrict__ sc,
                                                          int16_t* __restrict__ res, SResult* out) {
    const PDesc P = pd[blk_plane[blockIdx.x]];
    const SCall& C = sc[P.stream];
    if (!C.enc_on) return;
    const int key = C.enc_key;
    const bool mc = !key && sd[P.stream].mv_range > 0;   // residuals by k_mc_resid_b
    const int16_t* cur = C.ecur ? est1 : est0;
    int16_t* nxt = C.ecur ? est0 : est1;
    const QuantParams qp = sd[P.stream].qp;
    uint32_t* err = &out[P.stream].enc_err;
    const int total = (int)P.total, low_n = (int)P.low_n, low_w = P.low_w;
    const int base = (blockIdx.x - P.first_block) * ELEM_BLOCK + threadIdx.x;
    const float* cp = coef + P.coef_off;
    // every load of the thread first, so that they are in flight together
    float cv[ELEM_PER_THREAD], ca[ELEM_PER_THREAD];
    int pv[ELEM_PER_THREAD];
#pragma unroll
    for (int k = 0; k < ELEM_PER_THREAD; k++) {
        const int le = base + k * ELEM_THREADS;
        cv[k] = ca[k] = 0.f;
        pv[k] = 0;
        if (le >= total) continue;
        cv[k] = cp[le];
        if (!key) pv[k] = cur[P.coef_off + le];
        else if (le < low_n && le >= low_w) ca[k] = cp[le - low_w];
    }
#pragma unroll
    for (int k = 0; k < ELEM_PER_THREAD; k++) {
        const int le = base + k * ELEM_THREADS;
        if (le >= total) break;
        const long long e = P.coef_off + le;
        const bool low = le < low_n;
        const int q = quant(cv[k], low, qp, err);
        int r;
        if (!key) r = q - pv[k];
        else if (low && le >= low_w) r = q - quant(ca[k], true, qp, err);
        else r = q;
        nxt[e] = (int16_t)q;
        if (!mc) res[e] = (int16_t)(uint16_t)(r & 0xFFFF);   // wrapping 16-bit difference
    }
}

// decoder side: codes from residuals, then dequantised coefficients
__global__ void __launch_bounds__(ELEM_THREADS) k_unquant_b(const int16_t* __restrict__ res, int16_t* dst0,
                                                            int16_t* dst1, const PDesc* __restrict__ pd,
                                                            const int* __restrict__ blk_plane,
                                                            const SDesc* __restrict__ sd,
                                                            const SCall* __restrict__ sc,
                                                            const SResult* __restrict__ rs,
                                                            float* __restrict__ coef) {
    const PDesc P = pd[blk_plane[blockIdx.x]];
    const SCall& C = sc[P.stream];
    if (!C.dec_on || rs[P.stream].dec_err || rs[P.stream].dec_type == 2) return;   // type 2: k_mc_recon_b
    const bool key = rs[P.stream].dec_type == 0;
    const int16_t* cur = C.dcur ? dst1 : dst0;
    int16_t* nxt = C.dcur ? dst0 : dst1;
    const QuantParams qp = sd[P.stream].qp;
    const int total = (int)P.total, low_n = (int)P.low_n;
    const int base = (blockIdx.x - P.first_block) * ELEM_BLOCK + threadIdx.x;
#pragma unroll
    for (int k = 0; k < ELEM_PER_THREAD; k++) {
        const int le = base + k * ELEM_THREADS;
        if (le >= total) break;
        const bool low = le < low_n;
        if (key && low) continue;                   // column running sums: k_unquant_keylow_b
        const long long e = P.coef_off + le;
        const int q = key ? res[e] : (int16_t)(uint16_t)((res[e] + cur[e]) & 0xFFFF);
        nxt[e] = (int16_t)q;
        coef[e] = (float)q * (low ? qp.qpl_denorm : qp.qph);
    }
}

// K-frame lowpass: undo the column first difference (running sum down each column)
__global__ void k_unquant_keylow_b(const int16_t* __restrict__ res, int16_t* dst0, int16_t* dst1,
                                   const PDesc* __restrict__ pd, int nplanes, const SDesc* __restrict__ sd,
                                   const SCall* __restrict__ sc, const SResult* __restrict__ rs,
                                   float* __restrict__ coef) {
    int t = blockIdx.x * blockDim.x + threadIdx.x;
    for (int p = 0; p < nplanes; p++) {
        const PDesc P = pd[p];
        if (t >= P.low_w) {
            t -= P.low_w;
            continue;
        }
        const SCall& C = sc[P.stream];
        if (!C.dec_on || rs[P.stream].dec_err || rs[P.stream].dec_type != 0) return;
        const QuantParams qp = sd[P.stream].qp;
        const long long base = P.coef_off + t;
        const int rows = (int)(P.low_n / P.low_w);
        int acc = 0;
        for (int r = 0; r < rows; r++) {
            const long long e = base + (long long)r * P.low_w;
            acc = (int16_t)(uint16_t)((acc + res[e]) & 0xFFFF);
            (C.dcur ? dst0 : dst1)[e] = (int16_t)acc;
            coef[e] = (float)acc * qp.qpl_denorm;
        }
        return;
    }
}

// ------------------------------------------------------------- motion
// §3.2: full-search block matching of the padded luma plane in 16 x 16
// blocks against the previous frame's, over every displacement in
// [-W, W]^2 that keeps the block inside the plane.  The criterion is the sum
// of squared differences sum (c - p)^2 = sum c^2 + (sum p^2 - 2 sum c p); the
// first term is the same for every candidate of a block, so the search ranks
// the exact integer sum p^2 - 2 sum c p, with the same order and the same
// ties.  Ties go to the smaller |dy| + |dx|, then to the first candidate in
// raster order.  Full blocks use four-byte dot products of packed rows, a
// thread taking four neighbouring displacements (dx = 4g - W .. 4g - W + 3,
// one dy): the five window words of a row serve all four, shifted by a
// whole number of bytes known at compile time.
__global__ void __launch_bounds__(1024) k_motion_b(const SDesc* __restrict__ sd, const SCall* __restrict__ sc,
                                                  const int* __restrict__ blk_stream,
                                                  const uint8_t* __restrict__ luma0,
                                                  const uint8_t* __restrict__ luma1, int8_t* __restrict__ mv, int ws) {
    // the window, (16 + 2 W_max) rows of ws >= 16 + 2 W_max + 4 bytes, ws a multiple of 4 (W_max: the
    // batch's largest range)
    extern __shared__ __align__(16) uint8_t s_win[];
    __shared__ uint32_t s_cur[16 * 4];
    __shared__ unsigned long long s_best[32];
    const int s = blk_stream[blockIdx.x];
    const SCall& C = sc[s];
    if (!C.enc_on || C.enc_key) return;
    const SDesc& D = sd[s];
    const int R = D.mv_range, Hp = D.cg.Hp, Wp = D.cg.Wp;
    const int b = blockIdx.x - D.blk_motion;
    const int by = b / D.nbx, bx = b - by * D.nbx;
    const int y0 = 16 * by, x0 = 16 * bx;
    const int bh = min(16, Hp - y0), bw = min(16, Wp - x0);
    const uint8_t* cur = (C.ecur ? luma0 : luma1) + D.luma_off;    // this frame (written by the colour kernel)
    const uint8_t* prev = (C.ecur ? luma1 : luma0) + D.luma_off;
    // the window: previous-frame rows [y0 - R, y0 + bh + R), columns [x0 - R, x0 + bw + R),
    // in-plane bytes only (a valid candidate never reads the others)
    // a warp per window row, lanes along it
    const int nr = bh + 2 * R, nc = bw + 2 * R;
    const int lane = threadIdx.x & 31, nwarp = blockDim.x >> 5;
    for (int r = threadIdx.x >> 5; r < nr; r += nwarp) {
        const int gy = y0 - R + r;
        uint8_t* dst = s_win + r * ws;
        const bool row_in = gy >= 0 && gy < Hp;
        const uint8_t* src = prev + (long long)(row_in ? gy : 0) * Wp;
        for (int c = lane; c < nc; c += 32) {
            const int gx = x0 - R + c;
            dst[c] = (row_in && gx >= 0 && gx < Wp) ? src[gx] : 0;
        }
    }
    for (int t = threadIdx.x; t < 64; t += blockDim.x) {
        const int r = t >> 2, w = t & 3;
        uint32_t v = 0;
        for (int k = 0; k < 4; k++) {
            const int x = 4 * w + k;
            const uint32_t byte = (r < bh && x < bw) ? cur[(long long)(y0 + r) * Wp + x0 + x] : 0u;
            v |= byte << (8 * k);
        }
        s_cur[t] = v;
    }
    __syncthreads();
    const int side = 2 * R + 1;
    // key = (pp - 2 cp) + 2^26 (27 bits), then |dy| + |dx| (8 bits), then the raster index (15 bits)
    auto key_of = [&](unsigned cp, unsigned pp, int dy, int dx) {
        const int k = (dy + R) * side + (dx + R);
        return ((unsigned long long)(unsigned)((int)pp - 2 * (int)cp + (1 << 26)) << 23) |
               ((unsigned long long)(abs(dy) + abs(dx)) << 15) | (unsigned long long)k;
    };
    unsigned long long best = ~0ull;
    if (bw == 16) {
        // bytes are unsigned: the unsigned dot products.  Group g: dy = g / ngx - W, dx = 4 (g % ngx) - W + j;
        // its window words start at byte 4 (g % ngx) of the row (the last group may read up to
        // four bytes past the window's columns, inside the row stride: only for dx > W, never kept)
        const int ngx = (side + 3) >> 2, ng = side * ngx;
        for (int g = threadIdx.x; g < ng; g += blockDim.x) {
            const int gy = g / ngx, gx = g - gy * ngx;
            const int dy = gy - R, dx0 = 4 * gx - R;
            if (y0 + dy < 0 || y0 + dy + bh > Hp) continue;
            unsigned cp[4] = {0, 0, 0, 0}, pp[4] = {0, 0, 0, 0};
            const uint8_t* wbase = s_win + (dy + R) * ws + 4 * gx;
            for (int r = 0; r < bh; r++) {
                const uint32_t* wr = reinterpret_cast<const uint32_t*>(wbase + r * ws);
                uint32_t w[5], cw[4];
#pragma unroll
                for (int q = 0; q < 5; q++) w[q] = wr[q];
#pragma unroll
                for (int q = 0; q < 4; q++) cw[q] = s_cur[4 * r + q];
#pragma unroll
                for (int j = 0; j < 4; j++)
#pragma unroll
                    for (int q = 0; q < 4; q++) {
                        const uint32_t pw = j == 0 ? w[q] : __funnelshift_r(w[q], w[q + 1], 8 * j);
                        cp[j] = __dp4a(cw[q], pw, cp[j]);
                        pp[j] = __dp4a(pw, pw, pp[j]);
                    }
            }
#pragma unroll
            for (int j = 0; j < 4; j++) {
                const int dx = dx0 + j;
                if (dx > R || x0 + dx < 0 || x0 + dx + bw > Wp) continue;
                const unsigned long long key = key_of(cp[j], pp[j], dy, dx);
                best = key < best ? key : best;
            }
        }
    } else {
        const int ncand = side * side;
        for (int k = threadIdx.x; k < ncand; k += blockDim.x) {
            const int dy = k / side - R, dx = k - (k / side) * side - R;
            if (y0 + dy < 0 || y0 + dy + bh > Hp || x0 + dx < 0 || x0 + dx + bw > Wp) continue;
            unsigned cp = 0, pp = 0;
            const uint8_t* w0 = s_win + (dy + R) * ws + (dx + R);
            for (int r = 0; r < bh; r++)
                for (int x = 0; x < bw; x++) {
                    const unsigned p = w0[r * ws + x];
                    const unsigned c = (s_cur[4 * r + (x >> 2)] >> (8 * (x & 3))) & 255u;
                    cp += c * p;
                    pp += p * p;
                }
            const unsigned long long key = key_of(cp, pp, dy, dx);
            best = key < best ? key : best;
        }
    }
    for (int o = 16; o > 0; o >>= 1) {
        const unsigned long long other = __shfl_down_sync(0xffffffffu, best, o);
        best = other < best ? other : best;
    }
    if ((threadIdx.x & 31) == 0) s_best[threadIdx.x >> 5] = best;
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int w = 1; w < (int)(blockDim.x >> 5); w++) best = s_best[w] < best ? s_best[w] : best;
        best = s_best[0] < best ? s_best[0] : best;
        const int k = (int)(best & 0x7FFF);
        mv[2 * (D.mv_off + b)] = (int8_t)(k / side - R);
        mv[2 * (D.mv_off + b) + 1] = (int8_t)(k - (k / side) * side - R);
    }
}

// §3.7: the prediction of element (i, j) of a component from the previous
// codes: the vector of the luma block under luma sample (i 2^ey, j 2^ex),
// scaled by 2^-ey, 2^-ex (rounded half away from zero), clamped to the
// component
__device__ __forceinline__ int shift_round(int v, int e) {
    if (e == 0) return v;
    const int a = (abs(v) + (1 << (e - 1))) >> e;
    return v < 0 ? -a : a;
}

struct McRow {
    const int8_t* mvrow;   // the vectors of the block row under this component row
    long long base;        // global index of the component's first element
    int i, h, w, ey, ex, nbx;
};
// (one table load per row: the component's rows are contiguous, so its first
// element is the row's minus i rows)
__device__ __forceinline__ McRow mc_row(int row, const RowTable& rt, const SDesc& D, const int8_t* mv) {
    McRow m;
    const int4 t = rt.mc[row];
    m.i = t.x;
    m.h = t.y;
    m.w = rt.w[row];
    m.base = rt.off[row] - (long long)t.x * m.w;
    m.ey = t.z;
    m.ex = t.w;
    m.nbx = D.nbx;
    const int by = min((m.i << m.ey) >> 4, D.nby - 1);
    m.mvrow = mv + 2LL * by * D.nbx;
    return m;
}
__device__ __forceinline__ long long mc_src(const McRow& m, int x) {
    const int bx = min((x << m.ex) >> 4, m.nbx - 1);
    const int si = min(max(m.i + shift_round(m.mvrow[2 * bx], m.ey), 0), m.h - 1);
    const int sj = min(max(x + shift_round(m.mvrow[2 * bx + 1], m.ex), 0), m.w - 1);
    return m.base + (long long)si * m.w + sj;
}

// one warp per component row of the motion-compensated P-frames
__global__ void k_mc_resid_b(const int16_t* __restrict__ est0, const int16_t* __restrict__ est1, RowTable rt,
                             CompTable ct, const SDesc* __restrict__ sd, const SCall* __restrict__ sc,
                             const int8_t* __restrict__ mv, int16_t* __restrict__ res) {
    const int lane = threadIdx.x & 31;
    const int row = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (row >= rt.nrows) return;
    const int s = rt.stream[row];
    const SCall& C = sc[s];
    const SDesc& D = sd[s];
    if (!C.enc_on || C.enc_key || D.mv_range == 0) return;
    const int16_t* prev = C.ecur ? est1 : est0;
    const int16_t* q = C.ecur ? est0 : est1;       // this frame's codes (k_quant_b)
    const McRow m = mc_row(row, rt, D, mv + 2 * D.mv_off);
    const long long off = rt.off[row];
    // two elements per lane in flight: their gathers do not wait on each other
    for (int x = lane; x < m.w; x += 64) {
        const bool two = x + 32 < m.w;
        const long long s0 = mc_src(m, x), s1 = two ? mc_src(m, x + 32) : s0;
        const int16_t p0 = prev[s0], p1 = prev[s1], q0 = q[off + x];
        const int16_t q1 = two ? q[off + x + 32] : (int16_t)0;
        res[off + x] = (int16_t)(uint16_t)((q0 - p0) & 0xFFFF);
        if (two) res[off + x + 32] = (int16_t)(uint16_t)((q1 - p1) & 0xFFFF);
    }
}

__global__ void k_mc_recon_b(const int16_t* __restrict__ res, int16_t* dst0, int16_t* dst1, RowTable rt,
                             CompTable ct, const SDesc* __restrict__ sd, const SCall* __restrict__ sc,
                             const SResult* __restrict__ rs, float* __restrict__ coef) {
    const int lane = threadIdx.x & 31;
    const int row = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (row >= rt.nrows) return;
    const int s = rt.stream[row];
    const SCall& C = sc[s];
    if (!C.dec_on || rs[s].dec_err || rs[s].dec_type != 2) return;
    const SDesc& D = sd[s];
    const int16_t* prev = C.dcur ? dst1 : dst0;
    int16_t* nxt = C.dcur ? dst0 : dst1;
    const int8_t* v = reinterpret_cast<const int8_t*>(C.in + D.hdr_bytes + 2LL * rs[s].dec_tokens);
    const McRow m = mc_row(row, rt, D, v);
    const long long off = rt.off[row];
    const float scale = rt.low[row] ? D.qp.qpl_denorm : D.qp.qph;
    for (int x = lane; x < m.w; x += 64) {
        const bool two = x + 32 < m.w;
        const long long s0 = mc_src(m, x), s1 = two ? mc_src(m, x + 32) : s0;
        const int16_t p0 = prev[s0], p1 = prev[s1], r0 = res[off + x];
        const int16_t r1 = two ? res[off + x + 32] : (int16_t)0;
        const int16_t q0 = (int16_t)(uint16_t)((r0 + p0) & 0xFFFF);
        nxt[off + x] = q0;
        coef[off + x] = (float)q0 * scale;
        if (two) {
            const int16_t q1 = (int16_t)(uint16_t)((r1 + p1) & 0xFFFF);
            nxt[off + x + 32] = q1;
            coef[off + x + 32] = (float)q1 * scale;
        }
    }
}

// ------------------------------------------------------------------ RLE
// Rows of every component of every stream, in stream order.  Token count of
// a row: one per non-zero code plus two per maximal zero run; raw rows
// (K-frame lowpass) carry one token per code.
__global__ void k_rle_count_b(const int16_t* __restrict__ res, RowTable rt, const SCall* __restrict__ sc,
                              uint32_t* __restrict__ cnt) {
    const int lane = threadIdx.x & 31;
    const int row = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (row >= rt.nrows) return;
    const SCall& C = sc[rt.stream[row]];
    if (!C.enc_on) {
        if (lane == 0) cnt[row] = 0;
        return;
    }
    const long long off = rt.off[row];
    const int w = rt.w[row];
    if (C.enc_key && rt.low[row]) {
        if (lane == 0) cnt[row] = (uint32_t)w;
        return;
    }
    uint32_t n = 0;
    bool prev_zero = false;
    int16_t vn = lane < w ? res[off + lane] : (int16_t)1;     // the next chunk, loaded one chunk ahead
    for (int x0 = 0; x0 < w; x0 += 32) {
        int x = x0 + lane;
        bool valid = x < w;
        const int16_t v = vn;
        if (x + 32 < w) vn = res[off + x + 32];
        bool z = valid && v == 0;
        unsigned zb = __ballot_sync(0xffffffffu, z);
        unsigned vb = __ballot_sync(0xffffffffu, valid);
        unsigned starts = zb & ~((zb << 1) | (prev_zero ? 1u : 0u));
        n += __popc(vb & ~zb) + 2 * __popc(starts);
        prev_zero = (zb >> 31) & 1u;
    }
    if (lane == 0) cnt[row] = n;
}

__device__ __forceinline__ void put_tok(int16_t* tok, uint32_t pos, uint32_t cap_tok, int16_t v, uint32_t* err) {
    if (pos < cap_tok) tok[pos] = v;
    else atomicOr(err, EF_CAPACITY);
}

__global__ void k_rle_write_b(const int16_t* __restrict__ res, RowTable rt, const SDesc* __restrict__ sd,
                              const SCall* __restrict__ sc, const uint32_t* __restrict__ tokoff, SResult* out) {
    const int lane = threadIdx.x & 31;
    const int row = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (row >= rt.nrows) return;
    const int s = rt.stream[row];
    const SCall& C = sc[s];
    if (!C.enc_on) return;
    const SDesc& D = sd[s];
    if (C.out_cap < D.hdr_bytes) return;            // reported by the header kernel
    int16_t* tok = reinterpret_cast<int16_t*>(C.out + D.hdr_bytes);
    const long long capl = (C.out_cap - D.hdr_bytes) / 2;
    const uint32_t cap_tok = (uint32_t)(capl > 0xFFFFFFFFLL ? 0xFFFFFFFFLL : capl);
    uint32_t* err = &out[s].enc_err;
    const long long off = rt.off[row];
    const int w = rt.w[row];
    uint32_t pos = tokoff[row] - tokoff[D.row0];
    if (C.enc_key && rt.low[row]) {
        for (int x = lane; x < w; x += 32) put_tok(tok, pos + x, cap_tok, res[off + x], err);
        return;
    }
    const unsigned lt = (1u << lane) - 1u;
    bool prev_zero = false;
    uint32_t open_pos = 0;   // token position of the marker of a run left open by the previous chunk
    int open_x = 0;
    int16_t vn = lane < w ? res[off + lane] : (int16_t)1;     // the next chunk, loaded one chunk ahead
    for (int x0 = 0; x0 < w; x0 += 32) {
        int x = x0 + lane;
        bool valid = x < w;
        const int16_t v = valid ? vn : (int16_t)1;
        if (x + 32 < w) vn = res[off + x + 32];
        bool z = valid && v == 0;
        unsigned zb = __ballot_sync(0xffffffffu, z);
        unsigned vb = __ballot_sync(0xffffffffu, valid);
        unsigned starts = zb & ~((zb << 1) | (prev_zero ? 1u : 0u));
        unsigned nz = vb & ~zb;
        bool start = (starts >> lane) & 1u;
        uint32_t my = pos + __popc(nz & lt) + 2 * __popc(starts & lt);
        if (valid && !z) put_tok(tok, my, cap_tok, v, err);
        if (start) put_tok(tok, my, cap_tok, 0, err);
        // the run containing this lane started at the highest start lane <= lane, or before the chunk
        unsigned le = starts & (lt | (1u << lane));
        int sl = le ? 31 - __clz(le) : -1;
        uint32_t spos = __shfl_sync(0xffffffffu, my, sl < 0 ? 0 : sl);
        int sx = sl < 0 ? open_x : x0 + sl;
        if (sl < 0) spos = open_pos;
        // this lane ends its run if it is zero and the next element is not (or the row ends)
        // the element after lane 31 is the first of the next chunk (lane 0's prefetched value)
        const int16_t after = __shfl_sync(0xffffffffu, vn, 0);
        bool next_zero;
        if (lane < 31) next_zero = (zb >> (lane + 1)) & 1u;
        else next_zero = (x + 1 < w) && after == 0;
        if (z && !next_zero) put_tok(tok, spos + 1, cap_tok, (int16_t)(x - sx + 1), err);
        uint32_t spos31 = __shfl_sync(0xffffffffu, spos, 31);
        int sx31 = __shfl_sync(0xffffffffu, sx, 31);
        prev_zero = (zb >> 31) & 1u;
        if (prev_zero) {
            open_pos = spos31;
            open_x = sx31;
        }
        pos += __popc(nz) + 2 * __popc(starts);
    }
}

// one block per stream: header, component token counts, motion vectors, capacity check
__global__ void k_stream_header_b(const SDesc* __restrict__ sd, const SCall* __restrict__ sc,
                                  const uint32_t* __restrict__ tokoff, CompTable ct, const int8_t* __restrict__ mv,
                                  SResult* out) {
    const int s = blockIdx.x;
    const SCall& C = sc[s];
    if (!C.enc_on) return;
    const SDesc& D = sd[s];
    const uint32_t tokens = tokoff[D.row0 + D.nrows] - tokoff[D.row0];
    const bool mc = !C.enc_key && D.mv_range > 0;
    const long long need = D.hdr_bytes + 2LL * tokens + (mc ? D.mv_bytes : 0);
    if (threadIdx.x == 0) {
        out[s].enc_tokens = tokens;
        if (need > C.out_cap) atomicOr(&out[s].enc_err, EF_CAPACITY);
    }
    if (C.out_cap < D.hdr_bytes) return;
    uint8_t* o = C.out;
    if (threadIdx.x == 0) {
        const StreamHeader& h = D.hdr;
        o[0] = 'C'; o[1] = 'V'; o[2] = 'C'; o[3] = '1';
        o[4] = 1; o[5] = (uint8_t)h.flags;
        o[6] = (uint8_t)(C.enc_key ? 0 : (mc ? 2 : 1));
        o[7] = (uint8_t)h.levels;
        for (int i = 0; i < 4; i++) o[8 + i] = (uint8_t)(C.enc_index >> (8 * i));
        o[12] = (uint8_t)h.height; o[13] = (uint8_t)(h.height >> 8);
        o[14] = (uint8_t)h.width; o[15] = (uint8_t)(h.width >> 8);
        for (int i = 0; i < 6; i++) o[16 + i] = (uint8_t)h.dirs[i];
        o[22] = (uint8_t)h.qph; o[23] = (uint8_t)(h.qph >> 8);
        o[24] = (uint8_t)h.qpl; o[25] = (uint8_t)(h.qpl >> 8);
        o[26] = 0; o[27] = 0;
        for (int i = 0; i < 4; i++) o[28 + i] = (uint8_t)((unsigned)D.ncomp >> (8 * i));
    }
    for (int c = threadIdx.x; c < D.ncomp; c += blockDim.x) {
        const int g = D.comp0 + c;
        reinterpret_cast<uint32_t*>(o + 32)[c] = tokoff[ct.row0[g + 1]] - tokoff[ct.row0[g]];
    }
    // the vectors follow the tokens
    if (mc && need <= C.out_cap) {
        uint8_t* v = o + D.hdr_bytes + 2LL * tokens;
        const int8_t* m = mv + 2 * D.mv_off;
        for (long long i = threadIdx.x; i < D.mv_bytes; i += blockDim.x) v[i] = (uint8_t)m[i];
    }
}

// ------------------------------------------------------------ decoding
__device__ __forceinline__ uint32_t rd32(const uint8_t* p) {
    return (uint32_t)p[0] | ((uint32_t)p[1] << 8) | ((uint32_t)p[2] << 16) | ((uint32_t)p[3] << 24);
}
__device__ __forceinline__ int16_t rd16(const uint8_t* p) { return (int16_t)(uint16_t)(p[0] | (p[1] << 8)); }

__device__ __forceinline__ long long dec_in_len(const SDesc& D, const SCall& C, const SResult* enc, int s) {
    if (C.in_len >= 0) return C.in_len;
    if (enc[s].enc_err) return 0;
    // this call's encoder output
    return D.hdr_bytes + 2LL * enc[s].enc_tokens + (!C.enc_key && D.mv_range > 0 ? D.mv_bytes : 0);
}

// one block per stream: header check, component token offsets
__global__ void k_dec_parse_b(const SDesc* __restrict__ sd, const SCall* __restrict__ sc,
                              const SResult* __restrict__ enc, CompTable ct, uint32_t* __restrict__ comp_tok,
                              SResult* out) {
    const int s = blockIdx.x;
    const SCall& C = sc[s];
    __shared__ uint32_t s_carry;
    __shared__ int s_bad, s_drop;
    __shared__ uint32_t s_part[1024];
    if (!C.dec_on) {
        if (threadIdx.x == 0) out[s].dec_tokens = 0;
        return;
    }
    const SDesc& D = sd[s];
    const uint8_t* in = C.in;
    const long long in_len = dec_in_len(D, C, enc, s);
    const int ncomp = D.ncomp;
    if (threadIdx.x == 0) {
        int bad = 0;
        out[s].dec_type = 0;
        out[s].dec_tokens = 0;
        if (in_len < D.hdr_bytes) bad = EF_CORRUPT;
        else {
            const StreamHeader& e = D.hdr;
            if (in[0] != 'C' || in[1] != 'V' || in[2] != 'C' || in[3] != '1' || in[4] != 1 || in[5] > 5) bad = EF_CORRUPT;
            else if (in[5] != e.flags) bad = EF_MISMATCH;               // another storage or prototype
            int type = in[6];
            if (type > 2) bad = EF_CORRUPT;
            if (type == 2 && D.mv_range == 0) bad |= EF_MISMATCH;   // vectors for a decoder without motion
            if (in[7] != e.levels || (in[12] | (in[13] << 8)) != e.height || (in[14] | (in[15] << 8)) != e.width ||
                (in[22] | (in[23] << 8)) != e.qph || (in[24] | (in[25] << 8)) != e.qpl ||
                rd32(in + 28) != (uint32_t)ncomp)
                bad |= EF_MISMATCH;
            for (int i = 0; i < 6; i++)
                if (in[16 + i] != e.dirs[i]) bad |= EF_MISMATCH;
            uint32_t fidx = rd32(in + 8);
            if (!bad && type >= 1 && (C.dec_expect < 0 || (long long)fidx != C.dec_expect)) bad |= EF_STATE;
            // a frame without its finest `drop` levels serves scales >= drop; a P-frame
            // also needs the decoder state of the levels above the scale
            const int drop = in[26] | (in[27] << 8);
            if (drop > e.levels) bad |= EF_CORRUPT;
            if (!bad && (drop > C.dec_scale || (type >= 1 && C.dec_floor > C.dec_scale))) bad |= EF_STATE;
            out[s].dec_type = type;
            out[s].dec_index = fidx;
            out[s].dec_drop = bad ? 0 : (uint32_t)drop;
            s_drop = drop;
        }
        s_bad = bad;
        s_carry = 0;
    }
    __syncthreads();
    if (s_bad) {
        if (threadIdx.x == 0) out[s].dec_err |= (uint32_t)s_bad;
        return;
    }
    const int drop = s_drop;
    for (int base = 0; base < ncomp; base += blockDim.x) {
        int i = base + threadIdx.x;
        uint32_t v = i < ncomp ? rd32(in + 32 + 4 * i) : 0;
        if (v != 0 && i < ncomp) {
            const int lv = ct.level[D.comp0 + i];
            if (lv >= 1 && lv <= drop) atomicOr(&out[s].dec_err, EF_CORRUPT);   // dropped components hold no tokens
        }
        s_part[threadIdx.x] = v;
        __syncthreads();
        for (int d = 1; d < (int)blockDim.x; d <<= 1) {
            uint32_t a = threadIdx.x >= (unsigned)d ? s_part[threadIdx.x - d] : 0;
            __syncthreads();
            s_part[threadIdx.x] += a;
            __syncthreads();
        }
        if (i < ncomp) comp_tok[D.comp0 + i] = s_carry + s_part[threadIdx.x] - v;
        __syncthreads();
        if (threadIdx.x == blockDim.x - 1) s_carry += s_part[threadIdx.x];
        __syncthreads();
    }
    const uint32_t total = s_carry;
    const bool mc = out[s].dec_type == 2;
    const long long need = D.hdr_bytes + 2LL * total + (mc ? D.mv_bytes : 0);
    const bool ok = total != 0 && need <= in_len && total <= D.max_tok;   // a frame has tokens in its lowpass
    if (threadIdx.x == 0) {
        if (!ok) out[s].dec_err |= EF_CORRUPT;
        else out[s].dec_tokens = total;
    }
    // the vectors of a P-frame with motion lie within the search range
    if (ok && mc) {
        const int8_t* v = reinterpret_cast<const int8_t*>(in + D.hdr_bytes + 2LL * total);
        bool bad = false;
        for (long long i = threadIdx.x; i < D.mv_bytes; i += blockDim.x) bad |= v[i] < -D.mv_range || v[i] > D.mv_range;
        if (__syncthreads_or(bad) && threadIdx.x == 0) {
            out[s].dec_err |= EF_CORRUPT;
            out[s].dec_tokens = 0;
        }
    }
}

// exclusive scan of the streams' token counts: the base of each stream in
// the compact token space of this call; tok_base[n] = all tokens
__global__ void k_dec_base_b(const SDesc* __restrict__ sd, int nstreams, const SResult* __restrict__ rs,
                             uint32_t* __restrict__ tok_base) {
    (void)sd;
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    uint32_t acc = 0;
    for (int s = 0; s < nstreams; s++) {
        tok_base[s] = acc;
        acc += rs[s].dec_tokens;
    }
    tok_base[nstreams] = acc;
}

__device__ __forceinline__ int find_last_le(const uint32_t* a, int lo, int hi, uint32_t t) {
    // largest i in [lo, hi) with a[i] <= t (a non-decreasing, a[lo] <= t)
    while (hi - lo > 1) {
        int mid = (lo + hi) >> 1;
        if (a[mid] <= t) lo = mid;
        else hi = mid;
    }
    return lo;
}

// per token of the compact token space: stream, local index, component and its end
struct TokCtx {
    int s, c;
    uint32_t t, c0, c1;
};
__device__ __forceinline__ TokCtx tok_ctx(uint32_t g, const SDesc* sd, const SResult* rs, const uint32_t* tok_base,
                                          int nstreams, const uint32_t* comp_tok) {
    TokCtx k;
    // the stream whose range [tok_base[s], tok_base[s+1]) holds g (empty ranges skipped)
    int lo = 0, hi = nstreams;
    while (hi - lo > 1) {
        int mid = (lo + hi) >> 1;
        if (tok_base[mid] <= g) lo = mid;
        else hi = mid;
    }
    k.s = lo;
    const SDesc& D = sd[k.s];
    k.t = g - tok_base[k.s];
    k.c = find_last_le(comp_tok, D.comp0, D.comp0 + D.ncomp, k.t);
    k.c0 = comp_tok[k.c];
    k.c1 = (k.c + 1 < D.comp0 + D.ncomp) ? comp_tok[k.c + 1] : rs[k.s].dec_tokens;
    return k;
}

// elements produced by each token: value (and raw K-lowpass) tokens 1,
// zero markers 0, run counts n.  A thread takes TOK_GROUP consecutive tokens:
// one search for the first token's stream and component, then a forward walk.
constexpr int TOK_GROUP = 8;

__device__ __forceinline__ void tok_advance(TokCtx& k, uint32_t g, const SDesc* sd, const SResult* rs,
                                            const uint32_t* tok_base, int nstreams, const uint32_t* comp_tok) {
    // move k (valid for some g' < g) forward to token g
    while (k.s + 1 < nstreams && g >= tok_base[k.s + 1]) {
        k.s++;
        k.c = sd[k.s].comp0;
        k.c0 = comp_tok[k.c];
        const SDesc& D = sd[k.s];
        k.c1 = (k.c + 1 < D.comp0 + D.ncomp) ? comp_tok[k.c + 1] : rs[k.s].dec_tokens;
    }
    k.t = g - tok_base[k.s];
    const SDesc& D = sd[k.s];
    while (k.t >= k.c1 && k.c + 1 < D.comp0 + D.ncomp) {
        k.c++;
        k.c0 = k.c1;
        k.c1 = (k.c + 1 < D.comp0 + D.ncomp) ? comp_tok[k.c + 1] : rs[k.s].dec_tokens;
    }
}

__global__ void k_dec_contrib_b(const SDesc* __restrict__ sd, const SCall* __restrict__ sc,
                                const SResult* __restrict__ rs, const uint32_t* __restrict__ tok_base, int nstreams,
                                const uint32_t* __restrict__ comp_tok, CompTable ct, uint32_t* __restrict__ contrib,
                                SResult* out) {
    const uint32_t total = tok_base[nstreams];
    const uint32_t stride = gridDim.x * blockDim.x * TOK_GROUP;
    for (uint32_t g0 = (blockIdx.x * blockDim.x + threadIdx.x) * TOK_GROUP; g0 < total; g0 += stride) {
        TokCtx k = tok_ctx(g0, sd, rs, tok_base, nstreams, comp_tok);
        const uint32_t g1 = min(total, g0 + TOK_GROUP);
        for (uint32_t g = g0; g < g1; g++) {
            if (g > g0) tok_advance(k, g, sd, rs, tok_base, nstreams, comp_tok);
            const uint8_t* tok = sc[k.s].in + sd[k.s].hdr_bytes;
            const int16_t v = rd16(tok + 2LL * k.t);
            uint32_t n;
            if (rs[k.s].dec_type == 0 && ct.low[k.c]) n = 1;
            else if (k.t > k.c0 && rd16(tok + 2LL * (k.t - 1)) == 0) {
                n = v > 0 ? (uint32_t)v : 0;
                if (v <= 0) atomicOr(&out[k.s].dec_err, EF_CORRUPT);
            } else if (v != 0) n = 1;
            else {
                n = 0;
                if (k.t + 1 >= k.c1) atomicOr(&out[k.s].dec_err, EF_CORRUPT);
            }
            contrib[g] = n;
        }
    }
}

// The decoded codes of a frame that dropped its finest d levels are dense:
// each plane's lowpass, then its levels d+1..L.  Element offsets inside the
// stream: layout -> dense (for a component's first element) and back.
__device__ __forceinline__ long long absent_before(const SDesc& D, int d, int q) {
    long long a = 0;
    for (int i = 0; i < q; i++) a += D.absent[d][i];
    return a;
}
__device__ __forceinline__ long long dense_to_layout(const SDesc& D, int d, long long p) {
    const long long ds1 = D.pstart[1] - D.absent[d][0];
    const long long ds2 = D.pstart[2] - D.absent[d][0] - D.absent[d][1];
    const int q = p >= ds2 ? 2 : (p >= ds1 ? 1 : 0);
    const long long u = p - (q == 2 ? ds2 : (q == 1 ? ds1 : 0));
    return D.pstart[q] + (u < D.nlow[q] ? u : u + D.absent[d][q]);
}

// every component must expand to exactly its number of codes (none if dropped)
__global__ void k_dec_check_b(const SDesc* __restrict__ sd, const SResult* __restrict__ rs,
                              const uint32_t* __restrict__ tok_base, const uint32_t* __restrict__ comp_tok,
                              const uint32_t* __restrict__ pos, CompTable ct, SResult* out) {
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= ct.ncomp) return;
    const int s = ct.stream[c];
    if (rs[s].dec_tokens == 0) return;        // not decoding, or the header was rejected
    const SDesc& D = sd[s];
    const int d = min((int)rs[s].dec_drop, CVC_MAX_LEVELS);
    const int q = ct.plane[c], lv = ct.level[c];
    long long before = absent_before(D, d, q);
    if (lv >= 1 && lv <= d) before += ct.elem[c] - D.pstart[q] - D.nlow[q];
    else if (lv > d) before += D.absent[d][q];
    const uint32_t b = tok_base[s];
    const uint32_t p0 = pos[b];
    if ((long long)(pos[b + comp_tok[c]] - p0) != ct.elem[c] - before) atomicOr(&out[s].dec_err, EF_CORRUPT);
    if (c == D.comp0 + D.ncomp - 1 &&
        (long long)(pos[b + rs[s].dec_tokens] - p0) != D.ncoef - absent_before(D, d, 3))
        atomicOr(&out[s].dec_err, EF_CORRUPT);
}

__global__ void k_dec_scatter_b(const SDesc* __restrict__ sd, const SCall* __restrict__ sc,
                                const SResult* __restrict__ rs, const uint32_t* __restrict__ tok_base, int nstreams,
                                const uint32_t* __restrict__ comp_tok, CompTable ct, const uint32_t* __restrict__ pos,
                                int16_t* __restrict__ res) {
    const uint32_t total = tok_base[nstreams];
    const uint32_t stride = gridDim.x * blockDim.x * TOK_GROUP;
    for (uint32_t g0 = (blockIdx.x * blockDim.x + threadIdx.x) * TOK_GROUP; g0 < total; g0 += stride) {
        TokCtx k = tok_ctx(g0, sd, rs, tok_base, nstreams, comp_tok);
        const uint32_t g1 = min(total, g0 + TOK_GROUP);
        for (uint32_t g = g0; g < g1; g++) {
            if (g > g0) tok_advance(k, g, sd, rs, tok_base, nstreams, comp_tok);
            const SDesc& D = sd[k.s];
            const uint8_t* tok = sc[k.s].in + D.hdr_bytes;
            const int16_t v = rd16(tok + 2LL * k.t);
            const bool raw = rs[k.s].dec_type == 0 && ct.low[k.c];
            const bool count = !raw && k.t > k.c0 && rd16(tok + 2LL * (k.t - 1)) == 0;
            long long p = (long long)pos[g] - (long long)pos[tok_base[k.s]];
            const int d = min((int)rs[k.s].dec_drop, CVC_MAX_LEVELS);
            if (d > 0) p = dense_to_layout(D, d, p);
            if ((raw || (v != 0 && !count)) && p >= 0 && p < D.ncoef) res[D.coef_off + p] = v;
        }
    }
}

// ------------------------------------------------------ exclusive scans
constexpr int SCAN_CHUNK = 2048, SCAN_THREADS = 256;

__device__ __forceinline__ uint32_t block_reduce(uint32_t v, uint32_t* sh) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = v;
    __syncthreads();
    if (threadIdx.x < 32) {
        v = threadIdx.x < (blockDim.x >> 5) ? sh[threadIdx.x] : 0;
        for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    }
    return v;
}

// block b owns [b*chunk, min((b+1)*chunk, n)); n from the host or from device memory
__device__ __forceinline__ uint32_t scan_chunk(uint32_t n, const uint32_t* d_n) {
    return d_n ? ((n + gridDim.x - 1) / gridDim.x + 31) / 32 * 32 : SCAN_CHUNK;
}

__global__ void k_scan_reduce(const uint32_t* __restrict__ in, uint32_t n_host, const uint32_t* d_n,
                              uint32_t* __restrict__ sums) {
    __shared__ uint32_t sh[32];
    const uint32_t n = d_n ? *d_n : n_host;
    const uint32_t chunk = scan_chunk(n, d_n);
    const uint32_t base = blockIdx.x * chunk, end = min(base + chunk, n);
    uint32_t v = 0;
    for (uint32_t i = base + threadIdx.x; i < end; i += blockDim.x) v += in[i];
    v = block_reduce(v, sh);
    if (threadIdx.x == 0) sums[blockIdx.x] = v;
}

// in-place exclusive scan of the block sums (one block), total appended
__global__ void k_scan_sums(uint32_t* sums, int nb) {
    __shared__ uint32_t s[1024];
    __shared__ uint32_t carry;
    if (threadIdx.x == 0) carry = 0;
    __syncthreads();
    for (int base = 0; base < nb; base += blockDim.x) {
        int i = base + threadIdx.x;
        uint32_t v = i < nb ? sums[i] : 0;
        s[threadIdx.x] = v;
        __syncthreads();
        for (int d = 1; d < (int)blockDim.x; d <<= 1) {
            uint32_t a = threadIdx.x >= (unsigned)d ? s[threadIdx.x - d] : 0;
            __syncthreads();
            s[threadIdx.x] += a;
            __syncthreads();
        }
        if (i < nb) sums[i] = carry + s[threadIdx.x] - v;
        __syncthreads();
        if (threadIdx.x == blockDim.x - 1) carry += s[threadIdx.x];
        __syncthreads();
    }
    if (threadIdx.x == 0) sums[nb] = carry;
}

// each block scans its range in sub-chunks of SCAN_CHUNK (8 values per thread)
__global__ void __launch_bounds__(SCAN_THREADS) k_scan_apply(const uint32_t* __restrict__ in, uint32_t n_host, const uint32_t* d_n,
                             const uint32_t* __restrict__ sums, uint32_t* __restrict__ out) {
    __shared__ uint32_t wsum[32];
    __shared__ uint32_t s_carry;
    const uint32_t n = d_n ? *d_n : n_host;
    const uint32_t chunk = scan_chunk(n, d_n);
    const uint32_t base = blockIdx.x * chunk, end = min(base + chunk, n);
    constexpr int per = SCAN_CHUNK / SCAN_THREADS;   // a compile-time count keeps loc[] in registers
    if (threadIdx.x == 0) s_carry = sums[blockIdx.x];
    __syncthreads();
    for (uint32_t sub = base; sub < end; sub += SCAN_CHUNK) {
        uint32_t loc[per];
        uint32_t tsum = 0;
#pragma unroll
        for (int k = 0; k < per; k++) {
            uint32_t i = sub + threadIdx.x * per + k;
            loc[k] = i < end ? in[i] : 0;
            tsum += loc[k];
        }
        uint32_t x = tsum;
        for (int o = 1; o < 32; o <<= 1) {
            uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
            if ((threadIdx.x & 31) >= (unsigned)o) x += y;
        }
        if ((threadIdx.x & 31) == 31) wsum[threadIdx.x >> 5] = x;
        __syncthreads();
        if (threadIdx.x < 32) {
            uint32_t w = threadIdx.x < (blockDim.x >> 5) ? wsum[threadIdx.x] : 0;
            for (int o = 1; o < 32; o <<= 1) {
                uint32_t y = __shfl_up_sync(0xffffffffu, w, o);
                if (threadIdx.x >= (unsigned)o) w += y;
            }
            wsum[threadIdx.x] = w;
        }
        __syncthreads();
        uint32_t excl = s_carry + x - tsum + ((threadIdx.x >> 5) ? wsum[(threadIdx.x >> 5) - 1] : 0);
#pragma unroll
        for (int k = 0; k < per; k++) {
            uint32_t i = sub + threadIdx.x * per + k;
            if (i < end) out[i] = excl;
            excl += loc[k];
        }
        __syncthreads();
        if (threadIdx.x == 0) s_carry += wsum[(blockDim.x >> 5) - 1];
        __syncthreads();
    }
    if (blockIdx.x == gridDim.x - 1 && threadIdx.x == 0) out[n] = sums[gridDim.x];
}

cudaError_t exclusive_scan(const uint32_t* in, uint32_t n, uint32_t* out, uint32_t* tmp, cudaStream_t st) {
    int nb = (int)((n + SCAN_CHUNK - 1) / SCAN_CHUNK);
    if (nb == 0) nb = 1;
    k_scan_reduce<<<nb, 256, 0, st>>>(in, n, nullptr, tmp);
    k_scan_sums<<<1, 1024, 0, st>>>(tmp, nb);
    k_scan_apply<<<nb, SCAN_THREADS, 0, st>>>(in, n, nullptr, tmp, out);
    return cudaGetLastError();
}

cudaError_t exclusive_scan_dev(const uint32_t* in, const uint32_t* d_n, uint32_t n_max, uint32_t* out, uint32_t* tmp,
                               cudaStream_t st) {
    int nb = (int)std::min<uint32_t>(1024u, (n_max + SCAN_CHUNK - 1) / SCAN_CHUNK);
    if (nb < 1) nb = 1;
    k_scan_reduce<<<nb, 256, 0, st>>>(in, 0, d_n, tmp);
    k_scan_sums<<<1, 1024, 0, st>>>(tmp, nb);
    k_scan_apply<<<nb, SCAN_THREADS, 0, st>>>(in, 0, d_n, tmp, out);
    return cudaGetLastError();
}

}  // namespace cvc
