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

__global__ void __launch_bounds__(256, 8) k_colour_fwd_b(const SDesc* __restrict__ sd, const SCall* __restrict__ sc,
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
        // a thread takes two neighbouring chroma samples; where both average four whole source
        // pixels of aligned rows (2cx .. 2cx + 3: twelve bytes), it reads them as three words per row
        const bool rows4 = (((uintptr_t)r0 | (uintptr_t)r1) & 3) == 0;
        for (int cx = 2 * threadIdx.x; cx < g.Wcp; cx += 2 * blockDim.x) {
            uint32_t wd[2][3] = {{0u, 0u, 0u}, {0u, 0u, 0u}};   // source row: the bytes of pixels 2cx .. 2cx + 3
            const bool fast = rows4 && cx + 1 < g.Wc && 2 * cx + 3 < g.W;
            if (fast) {
#pragma unroll
                for (int r = 0; r < 2; r++) {
                    const uint32_t* w = reinterpret_cast<const uint32_t*>((r ? r1 : r0) + 6 * cx);
                    wd[r][0] = w[0];
                    wd[r][1] = w[1];
                    wd[r][2] = w[2];
                }
            }
#pragma unroll
            for (int h = 0; h < 2; h++) {
                const int c = cx + h;
                int sco = 0, scg = 0;
                const int sx = mirror_idx(c, g.Wc);
                const int c0 = 3 * (2 * sx), c1 = 3 * min(2 * sx + 1, g.W - 1);
                const uint8_t* q[4] = {r0 + c0, r0 + c1, r1 + c0, r1 + c1};
#pragma unroll
                for (int k = 0; k < 4; k++) {
                    // pixel k: source row k >> 1, column 2c + (k & 1)
                    const int o = 6 * h + 3 * (k & 1);
                    int R, G, Bv;
                    if (fast) {
                        R = (int)((wd[k >> 1][o >> 2] >> (8 * (o & 3))) & 255u);
                        G = (int)((wd[k >> 1][(o + 1) >> 2] >> (8 * ((o + 1) & 3))) & 255u);
                        Bv = (int)((wd[k >> 1][(o + 2) >> 2] >> (8 * ((o + 2) & 3))) & 255u);
                    } else {
                        R = q[k][0];
                        G = q[k][1];
                        Bv = q[k][2];
                    }
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
                oco[c] = (float)((sco + 2) >> 2);
                ocg[c] = (float)((scg + 2) >> 2);
            }
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
// POW2: every step of the launch is a power of two (no division in the kernel)
template <bool POW2 = false>
__device__ __forceinline__ int quant(float c, bool low, const QuantParams& q, uint32_t* err) {
    float t;
    if (low) t = c * q.low_scale;                    // exact power-of-two normalisation
    else t = (fabsf(c) >= q.threshold) ? c : 0.0f;
    // the IEEE quotient t / QP, ties away from zero; for a power-of-two QP the product with
    // its exact reciprocal is that same correctly rounded quotient
    const float r = low ? q.rqpl : q.rqph;
    float v = roundf(POW2 || r != 0.0f ? t * r : t / (low ? q.qpl : q.qph));
    // 8-bit storage (§3.6): the rounded code is kept in a byte
    if (q.st8) v = low ? fminf(fmaxf(v, 0.0f), 255.0f) : fminf(fmaxf(v, -128.0f), 127.0f);
    if (!(fabsf(v) <= 32767.0f)) {
        atomicOr(err, EF_OVERFLOW);
        return 0;
    }
    return (int)v;
}

// codes q (the next coder state) and residuals r of one frame per stream;
// a block covers ELEM_BLOCK elements of one plane, ELEM_PER_THREAD per thread.
// Planes whose coefficients start on a 4-element boundary (all but odd layouts)
// move runs of 4 consecutive elements with 16-byte float and 8-byte code
// accesses: thread t takes elements 4t .. 4t + 3 and 4(t + ELEM_THREADS) ..
// of its block; a ragged tail and a key frame's lowpass predictions go element
// by element.  Every element takes the same operations either way.
constexpr int ELEM_VEC = ELEM_PER_THREAD / 4;
static_assert(ELEM_PER_THREAD % 4 == 0, "runs of four");

__device__ __forceinline__ void unpack4(uint2 w, int* v) {
    v[0] = (int16_t)(w.x & 0xFFFF);
    v[1] = (int16_t)(w.x >> 16);
    v[2] = (int16_t)(w.y & 0xFFFF);
    v[3] = (int16_t)(w.y >> 16);
}
__device__ __forceinline__ uint2 pack4(const int* v) {
    return make_uint2((uint32_t)(v[0] & 0xFFFF) | ((uint32_t)v[1] << 16), (uint32_t)(v[2] & 0xFFFF) | ((uint32_t)v[3] << 16));
}
__device__ __forceinline__ bool vec_ok(long long e0, const void* a, const void* b, const void* c, const void* d) {
    return (e0 & 3) == 0 && ((reinterpret_cast<uintptr_t>(a) | reinterpret_cast<uintptr_t>(b) |
                              reinterpret_cast<uintptr_t>(c) | reinterpret_cast<uintptr_t>(d)) & 15) == 0;
}

template <bool POW2>
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
    const float* cp = coef + P.coef_off;
    if (vec_ok(P.coef_off, coef, est0, est1, res)) {
        const int blk0 = (blockIdx.x - P.first_block) * ELEM_BLOCK;
        // every load of the thread first, so that they are in flight together
        float4 cv[ELEM_VEC];
        uint2 pv[ELEM_VEC];
#pragma unroll
        for (int k = 0; k < ELEM_VEC; k++) {
            const int le = blk0 + 4 * (threadIdx.x + k * ELEM_THREADS);
            cv[k] = make_float4(0.f, 0.f, 0.f, 0.f);
            pv[k] = make_uint2(0u, 0u);
            if (le + 4 > total) continue;
            cv[k] = *reinterpret_cast<const float4*>(cp + le);
            if (!key) pv[k] = *reinterpret_cast<const uint2*>(cur + P.coef_off + le);
        }
#pragma unroll
        for (int k = 0; k < ELEM_VEC; k++) {
            const int le = blk0 + 4 * (threadIdx.x + k * ELEM_THREADS);
            if (le >= total) break;
            const bool whole = le + 4 <= total;
            float c[4] = {cv[k].x, cv[k].y, cv[k].z, cv[k].w};
            int pr[4], q[4], r[4];
            unpack4(pv[k], pr);
#pragma unroll
            for (int j = 0; j < 4; j++) {
                const int lj = le + j;
                q[j] = r[j] = 0;
                if (lj >= total) continue;
                if (!whole) {
                    c[j] = cp[lj];
                    if (!key) pr[j] = cur[P.coef_off + lj];
                }
                const bool low = lj < low_n;
                q[j] = quant<POW2>(c[j], low, qp, err);
                if (!key) r[j] = q[j] - pr[j];
                else if (low && lj >= low_w) r[j] = q[j] - quant<POW2>(cp[lj - low_w], true, qp, err);
                else r[j] = q[j];
            }
            const long long e = P.coef_off + le;
            if (whole) {
                *reinterpret_cast<uint2*>(nxt + e) = pack4(q);
                if (!mc) *reinterpret_cast<uint2*>(res + e) = pack4(r);   // wrapping 16-bit differences
            } else {
#pragma unroll
                for (int j = 0; j < 4; j++) {
                    if (le + j >= total) break;
                    nxt[e + j] = (int16_t)q[j];
                    if (!mc) res[e + j] = (int16_t)(uint16_t)(r[j] & 0xFFFF);
                }
            }
        }
        return;
    }
    const int base = (blockIdx.x - P.first_block) * ELEM_BLOCK + threadIdx.x;
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
        const int q = quant<POW2>(cv[k], low, qp, err);
        int r;
        if (!key) r = q - pv[k];
        else if (low && le >= low_w) r = q - quant<POW2>(ca[k], true, qp, err);
        else r = q;
        nxt[e] = (int16_t)q;
        if (!mc) res[e] = (int16_t)(uint16_t)(r & 0xFFFF);   // wrapping 16-bit difference
    }
}

// decoder side: codes from residuals, then dequantised coefficients (runs of four
// elements as in k_quant_b where the plane's layout allows)
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
    if (vec_ok(P.coef_off, res, dst0, dst1, coef)) {
        const int blk0 = (blockIdx.x - P.first_block) * ELEM_BLOCK;
        uint2 rv[ELEM_VEC], cv[ELEM_VEC];
#pragma unroll
        for (int k = 0; k < ELEM_VEC; k++) {
            const int le = blk0 + 4 * (threadIdx.x + k * ELEM_THREADS);
            rv[k] = cv[k] = make_uint2(0u, 0u);
            if (le + 4 > total || (key && le < low_n)) continue;
            rv[k] = *reinterpret_cast<const uint2*>(res + P.coef_off + le);
            if (!key) cv[k] = *reinterpret_cast<const uint2*>(cur + P.coef_off + le);
        }
#pragma unroll
        for (int k = 0; k < ELEM_VEC; k++) {
            const int le = blk0 + 4 * (threadIdx.x + k * ELEM_THREADS);
            if (le >= total) break;
            const long long e = P.coef_off + le;
            if (le + 4 > total || (key && le < low_n)) {
                // a ragged tail, or a run touching a key frame's lowpass (k_unquant_keylow_b's)
#pragma unroll
                for (int j = 0; j < 4; j++) {
                    const int lj = le + j;
                    if (lj >= total) break;
                    const bool low = lj < low_n;
                    if (key && low) continue;
                    const int q = key ? res[e + j] : (int16_t)(uint16_t)((res[e + j] + cur[e + j]) & 0xFFFF);
                    nxt[e + j] = (int16_t)q;
                    coef[e + j] = (float)q * (low ? qp.qpl_denorm : qp.qph);
                }
                continue;
            }
            int r[4], c[4], q[4];
            unpack4(rv[k], r);
            unpack4(cv[k], c);
            float f[4];
#pragma unroll
            for (int j = 0; j < 4; j++) {
                q[j] = key ? r[j] : (int16_t)(uint16_t)((r[j] + c[j]) & 0xFFFF);
                f[j] = (float)q[j] * (le + j < low_n ? qp.qpl_denorm : qp.qph);
            }
            *reinterpret_cast<uint2*>(nxt + e) = pack4(q);
            *reinterpret_cast<float4*>(coef + e) = make_float4(f[0], f[1], f[2], f[3]);
        }
        return;
    }
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
// Work units are tiles: runs of whole rows of one component (all of width w),
// in stream order, of at most RLE_TILE codes unless one row is longer.  A
// row's tokens (§3.8): one per non-zero code and two (0, n) per maximal zero
// run; the rows of a K-frame lowpass are stored raw, one token per code.
// A token's position in its stream is the exclusive scan of the tiles' token
// counts plus its place inside the tile, so the rows of a tile need no table.
//
// A thread takes 8 consecutive codes (one 16-byte load) and describes them by
// bit masks: inside the tile, non-zero, start and end of a zero run (a zero
// whose predecessor, resp. successor, in the row is non-zero or absent).

struct RleChunk {
    uint32_t w[4];          // the 8 codes, two per word, low half first
    unsigned nz, rs, re;    // non-zero codes, zero-run starts, zero-run ends (inside the tile)
};

__device__ __forceinline__ int16_t chunk_code(const RleChunk& k, int j) {
    const uint32_t v = (j & 4) ? ((j & 2) ? k.w[3] : k.w[2]) : ((j & 2) ? k.w[1] : k.w[0]);
    return (int16_t)(uint16_t)((j & 1) ? (v >> 16) : (v & 0xFFFFu));
}

// the codes g .. g+7 (g a multiple of 8, g + 8 > e0) of the tile [e0, e1) of rows of width w
__device__ __forceinline__ RleChunk rle_chunk(const int16_t* __restrict__ res, long long g, long long e0, long long e1,
                                              int w) {
    RleChunk k;
    const int4 v = *reinterpret_cast<const int4*>(res + g);
    k.w[0] = (uint32_t)v.x;
    k.w[1] = (uint32_t)v.y;
    k.w[2] = (uint32_t)v.z;
    k.w[3] = (uint32_t)v.w;
    const int rel = (int)(g - e0);                 // tile index of code 0 (negative in the first chunk)
    const int jf = rel < 0 ? -rel : 0;             // first code inside the tile
    const int jl = (int)min(8LL, e1 - g);          // one past the last
    const unsigned valid = (jl > jf ? (1u << jl) - (1u << jf) : 0u);
    unsigned zero = 0;
#pragma unroll
    for (int q = 0; q < 4; q++) {
        const uint32_t z = __vcmpeq2(k.w[q], 0u);  // 0xFFFF per zero half
        zero |= ((z & 1u) | ((z >> 15) & 2u)) << (2 * q);
    }
    zero &= valid;
    // row starts and ends among codes jf .. 7; code jf sits at row position p0
    const int p0 = (rel + jf) % w;
    unsigned rstart = 0, rend = 0;
    if (w >= 8) {
        const int js = jf + (p0 == 0 ? 0 : w - p0), je = jf + w - 1 - p0;
        rstart = js < 8 ? 1u << js : 0u;
        rend = je < 8 ? 1u << je : 0u;
    } else {
        int p = p0;
#pragma unroll
        for (int j = 0; j < 8; j++) {
            if (j >= jf) {
                rstart |= (p == 0 ? 1u : 0u) << j;
                rend |= (p == w - 1 ? 1u : 0u) << j;
                p = p + 1 == w ? 0 : p + 1;
            }
        }
    }
    // the codes just outside the chunk, where they are in the tile
    const bool zprev = jf == 0 && rel > 0 && res[g - 1] == 0;
    const bool znext = g + 8 < e1 && res[g + 8] == 0;
    const unsigned zp = (zero << 1) | (zprev ? 1u : 0u);   // zero-ness of each code's predecessor
    const unsigned zn = (zero >> 1) | (znext ? 0x80u : 0u); // ... and successor
    k.nz = valid & ~zero;
    k.rs = zero & (rstart | ~zp);
    k.re = zero & (rend | ~zn);
    return k;
}

__device__ __forceinline__ bool rle_raw(const SCall& C, const RleTiles& tt, int tile) {
    return C.enc_key && tt.low[tile];
}

__global__ void __launch_bounds__(RLE_THREADS) k_rle_count_b(const int16_t* __restrict__ res, RleTiles tt,
                                                              const SCall* __restrict__ sc, uint32_t* __restrict__ cnt) {
    __shared__ uint32_t s_part[RLE_THREADS / 32];
    const int tile = blockIdx.x;
    const SCall& C = sc[tt.stream[tile]];
    const long long e0 = tt.off[tile];
    const int n = tt.n[tile];
    if (!C.enc_on || rle_raw(C, tt, tile)) {
        if (threadIdx.x == 0) cnt[tile] = C.enc_on ? (uint32_t)n : 0u;
        return;
    }
    const long long e1 = e0 + n;
    const int w = tt.w[tile];
    uint32_t c = 0;
    for (long long g = (e0 & ~7LL) + 8LL * threadIdx.x; g < e1; g += RLE_CHUNK) {
        const RleChunk k = rle_chunk(res, g, e0, e1, w);
        c += __popc(k.nz) + 2 * __popc(k.rs);
    }
    for (int o = 16; o > 0; o >>= 1) c += __shfl_down_sync(0xffffffffu, c, o);
    if ((threadIdx.x & 31) == 0) s_part[threadIdx.x >> 5] = c;
    __syncthreads();
    if (threadIdx.x == 0) {
        uint32_t t = 0;
#pragma unroll
        for (int i = 0; i < RLE_THREADS / 32; i++) t += s_part[i];
        cnt[tile] = t;
    }
}

__global__ void __launch_bounds__(RLE_THREADS) k_rle_write_b(const int16_t* __restrict__ res, RleTiles tt,
                                                              const SDesc* __restrict__ sd, const SCall* __restrict__ sc,
                                                              const uint32_t* __restrict__ tileoff, SResult* out) {
    // warp totals of a chunk, double-buffered: chunk c + 1 writes the other half, so one
    // barrier per chunk separates every write from the reads of the same half
    __shared__ uint32_t s_sum[2][RLE_THREADS / 32];
    __shared__ int s_max[2][RLE_THREADS / 32];
    const int tile = blockIdx.x;
    const int s = tt.stream[tile];
    const SCall& C = sc[s];
    if (!C.enc_on) return;
    const SDesc& D = sd[s];
    if (C.out_cap < D.hdr_bytes) return;            // reported by the header kernel
    int16_t* tok = reinterpret_cast<int16_t*>(C.out + D.hdr_bytes);
    const long long capl = (C.out_cap - D.hdr_bytes) / 2;
    const uint32_t cap_tok = (uint32_t)(capl > 0xFFFFFFFFLL ? 0xFFFFFFFFLL : capl);
    const long long e0 = tt.off[tile];
    const int n = tt.n[tile];
    const uint32_t pos0 = tileoff[tile] - tileoff[D.tile0];
    bool over = false;
    if (rle_raw(C, tt, tile)) {
        for (int x = threadIdx.x; x < n; x += RLE_THREADS) {
            const uint32_t p = pos0 + x;
            if (p < cap_tok) tok[p] = res[e0 + x];
            else over = true;
        }
    } else {
        const long long e1 = e0 + n;
        const int w = tt.w[tile];
        const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
        uint32_t carry = 0;     // tokens of the tile's earlier chunks
        int carry_s = -1;       // latest zero-run start among them (tile index)
        int half = 0;
        for (long long gb = e0 & ~7LL; gb < e1; gb += RLE_CHUNK, half ^= 1) {
            const long long g = gb + 8LL * threadIdx.x;
            RleChunk k;
            if (g < e1) k = rle_chunk(res, g, e0, e1, w);
            else k.nz = k.rs = k.re = 0u;
            const int rel = (int)(g - e0);
            const uint32_t cn = __popc(k.nz) + 2 * __popc(k.rs);
            const int ls = k.rs ? rel + 31 - __clz(k.rs) : -1;
            // block scans: exclusive token offset, latest run start before this chunk
            uint32_t x = cn;
            int mx = ls;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
                const int ym = __shfl_up_sync(0xffffffffu, mx, o);
                if (lane >= o) {
                    x += y;
                    mx = max(mx, ym);
                }
            }
            int mprev = __shfl_up_sync(0xffffffffu, mx, 1);
            if (lane == 0) mprev = -1;
            if (lane == 31) {
                s_sum[half][warp] = x;
                s_max[half][warp] = mx;
            }
            __syncthreads();
            uint32_t wpre = 0, tot = 0;
            int wmax = -1, bmax = -1;
#pragma unroll
            for (int i = 0; i < RLE_THREADS / 32; i++) {
                const uint32_t a = s_sum[half][i];
                const int b = s_max[half][i];
                if (i < warp) {
                    wpre += a;
                    wmax = max(wmax, b);
                }
                tot += a;
                bmax = max(bmax, b);
            }
            const uint32_t tpos = pos0 + carry + wpre + x - cn;
            const int sprev = max(carry_s, max(wmax, mprev));
            unsigned m = k.nz | k.rs | k.re;
            while (m) {
                const int j = __ffs(m) - 1;
                m &= m - 1;
                const unsigned bit = 1u << j, below = bit - 1u;
                const uint32_t pj = tpos + __popc(k.nz & below) + 2 * __popc(k.rs & below);
                uint32_t p1 = pj, p2 = 0xFFFFFFFFu;
                int16_t v1 = 0, v2 = 0;
                if (k.nz & bit) v1 = chunk_code(k, j);   // a non-zero code, or a run's marker (0)
                if (k.re & bit) {
                    // the count of the run this code ends, after the run's marker
                    const unsigned le = k.rs & (below | bit);
                    const int sr = le ? rel + 31 - __clz(le) : sprev;
                    const int er = rel + j;
                    p2 = sr == er ? pj + 1 : pj - 1;
                    v2 = (int16_t)(er - sr + 1);
                    if (!(k.rs & bit)) p1 = 0xFFFFFFFFu;   // a run's last code writes only its count
                }
                if (p1 != 0xFFFFFFFFu) {
                    if (p1 < cap_tok) tok[p1] = v1;
                    else over = true;
                }
                if (p2 != 0xFFFFFFFFu) {
                    if (p2 < cap_tok) tok[p2] = v2;
                    else over = true;
                }
            }
            carry += tot;
            carry_s = max(carry_s, bmax);
        }
    }
    if (over) atomicOr(&out[s].enc_err, EF_CAPACITY);
}

// one block per stream: header, component token counts, motion vectors, capacity check
__global__ void k_stream_header_b(const SDesc* __restrict__ sd, const SCall* __restrict__ sc,
                                  const uint32_t* __restrict__ tileoff, CompTable ct, const int8_t* __restrict__ mv,
                                  SResult* out) {
    const int s = blockIdx.x;
    const SCall& C = sc[s];
    if (!C.enc_on) return;
    const SDesc& D = sd[s];
    const uint32_t tokens = tileoff[D.tile0 + D.ntiles] - tileoff[D.tile0];
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
        reinterpret_cast<uint32_t*>(o + 32)[c] = tileoff[ct.tile0[g + 1]] - tileoff[ct.tile0[g]];
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

// Token tiles of the decoder: every stream's tokens cut into tiles of
// DEC_TILE (a stream's last tile may be short), numbered stream after stream.
// k_dec_base_b: per stream the first token of the call's compact token space
// and the first tile; tile_base[n] = all tiles.
__global__ void k_dec_base_b(const SDesc* __restrict__ sd, int nstreams, const SResult* __restrict__ rs,
                             uint32_t* __restrict__ tok_base, uint32_t* __restrict__ tile_base) {
    (void)sd;
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    uint32_t acc = 0, tiles = 0;
    for (int s = 0; s < nstreams; s++) {
        tok_base[s] = acc;
        tile_base[s] = tiles;
        acc += rs[s].dec_tokens;
        tiles += (rs[s].dec_tokens + DEC_TILE - 1) / DEC_TILE;
    }
    tok_base[nstreams] = acc;
    tile_base[nstreams] = tiles;
}

// The DEC_PER_THREAD tokens of one thread: values, codes produced (raw and
// value tokens one, counts n, markers none), component of each token, and
// whether the group broke a rule of the format.
struct DecGroup {
    int16_t v[DEC_PER_THREAD];
    uint32_t n[DEC_PER_THREAD];
    int comp[DEC_PER_THREAD];     // global component index; -1 past the stream's last token
    bool code[DEC_PER_THREAD];    // the token is a code (raw or non-zero value) to place
    bool bad;
};

// the tile's stream (thread 0 searches; the block reads it from shared memory)
__device__ __forceinline__ int dec_tile_stream(const uint32_t* tile_base, int nstreams, int tile, int* s_sh) {
    if (threadIdx.x == 0) {
        int lo = 0, hi = nstreams;   // largest s with tile_base[s] <= tile (skips streams without tiles)
        while (hi - lo > 1) {
            const int mid = (lo + hi) >> 1;
            if (tile_base[mid] <= (uint32_t)tile) lo = mid;
            else hi = mid;
        }
        *s_sh = lo;
    }
    __syncthreads();
    return *s_sh;
}

// tokens t0 .. t0 + DEC_PER_THREAD - 1 of stream s (t0 a multiple of DEC_PER_THREAD);
// ctok: the stream's component token offsets in shared memory (ncomp of them)
__device__ __forceinline__ DecGroup dec_group(const uint8_t* tok, uint32_t t0, uint32_t ntok, const uint32_t* ctok,
                                              int ncomp, int comp0, bool key, const CompTable& ct) {
    DecGroup G;
    G.bad = false;
    // the group's values (4-byte loads where the token array allows them)
    if ((reinterpret_cast<uintptr_t>(tok) & 3) == 0) {
        const uint32_t* w = reinterpret_cast<const uint32_t*>(tok + 2ull * t0);
#pragma unroll
        for (int k = 0; k < DEC_PER_THREAD / 2; k++) {
            // the word of the stream's last token may reach 2 bytes past it, inside that aligned word
            const uint32_t x = t0 + 2 * k < ntok ? w[k] : 0u;
            G.v[2 * k] = (int16_t)(uint16_t)(x & 0xFFFFu);
            G.v[2 * k + 1] = (int16_t)(uint16_t)(x >> 16);
        }
    } else {
#pragma unroll
        for (int k = 0; k < DEC_PER_THREAD; k++) G.v[k] = t0 + k < ntok ? rd16(tok + 2ull * (t0 + k)) : (int16_t)0;
    }
    int16_t prev = t0 > 0 ? rd16(tok + 2ull * (t0 - 1)) : (int16_t)1;
    // the component of t0: largest c with ctok[c] <= t0
    int lo = 0, hi = ncomp;
    while (hi - lo > 1) {
        const int mid = (lo + hi) >> 1;
        if (ctok[mid] <= t0) lo = mid;
        else hi = mid;
    }
    int c = lo;
    uint32_t c0 = ctok[c], c1 = c + 1 < ncomp ? ctok[c + 1] : ntok;
#pragma unroll
    for (int k = 0; k < DEC_PER_THREAD; k++) {
        const uint32_t t = t0 + k;
        G.n[k] = 0;
        G.code[k] = false;
        G.comp[k] = -1;
        if (t < ntok) {
            while (t >= c1 && c + 1 < ncomp) {
                c++;
                c0 = c1;
                c1 = c + 1 < ncomp ? ctok[c + 1] : ntok;
            }
            G.comp[k] = comp0 + c;
            const int16_t v = G.v[k];
            if (key && ct.low[comp0 + c]) {
                G.n[k] = 1;                      // a K-frame lowpass code, stored raw
                G.code[k] = true;
            } else if (t > c0 && prev == 0) {
                // the count of the zero run opened by the previous token
                if (v > 0) G.n[k] = (uint32_t)v;
                else G.bad = true;
            } else if (v != 0) {
                G.n[k] = 1;
                G.code[k] = true;
            } else if (t + 1 >= c1) {
                G.bad = true;                    // a run marker without its count
            }
        }
        prev = G.v[k];
    }
    return G;
}

// codes produced by every token tile (a grid-stride loop over the call's tiles)
__global__ void __launch_bounds__(DEC_THREADS) k_dec_count_b(const SDesc* __restrict__ sd,
                                                              const SCall* __restrict__ sc,
                                                              const SResult* __restrict__ rs,
                                                              const uint32_t* __restrict__ tile_base, int nstreams,
                                                              const uint32_t* __restrict__ comp_tok, CompTable ct,
                                                              uint32_t* __restrict__ tile_sum, SResult* out) {
    __shared__ int s_stream;
    __shared__ uint32_t s_part[DEC_THREADS / 32];
    __shared__ uint32_t s_ctok[DEC_MAX_COMP];
    const int ntiles = (int)tile_base[nstreams];
    for (int tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
        const int s = dec_tile_stream(tile_base, nstreams, tile, &s_stream);
        const SDesc& D = sd[s];
        for (int i = threadIdx.x; i < D.ncomp; i += DEC_THREADS) s_ctok[i] = comp_tok[D.comp0 + i];
        __syncthreads();
        const uint32_t ntok = rs[s].dec_tokens;
        const uint32_t t0 = (uint32_t)(tile - (int)tile_base[s]) * DEC_TILE + DEC_PER_THREAD * threadIdx.x;
        uint32_t sum = 0;
        bool bad = false;
        if (t0 < ntok) {
            const DecGroup G = dec_group(sc[s].in + D.hdr_bytes, t0, ntok, s_ctok, D.ncomp, D.comp0,
                                         rs[s].dec_type == 0, ct);
#pragma unroll
            for (int k = 0; k < DEC_PER_THREAD; k++) sum += G.n[k];
            bad = G.bad;
        }
        if (bad) atomicOr(&out[s].dec_err, EF_CORRUPT);
        for (int o = 16; o > 0; o >>= 1) sum += __shfl_down_sync(0xffffffffu, sum, o);
        if ((threadIdx.x & 31) == 0) s_part[threadIdx.x >> 5] = sum;
        __syncthreads();
        if (threadIdx.x == 0) {
            uint32_t t = 0;
#pragma unroll
            for (int i = 0; i < DEC_THREADS / 32; i++) t += s_part[i];
            tile_sum[tile] = t;
        }
        __syncthreads();   // shared arrays are reused by the next tile
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

// every token tile again: the position of each code (its tile's exclusive
// prefix inside the stream plus a block scan), the codes placed into the
// zeroed residual frame, and the codes of each component summed for the check
__global__ void __launch_bounds__(DEC_THREADS) k_dec_scatter_b(const SDesc* __restrict__ sd,
                                                                const SCall* __restrict__ sc,
                                                                const SResult* __restrict__ rs,
                                                                const uint32_t* __restrict__ tile_base, int nstreams,
                                                                const uint32_t* __restrict__ comp_tok, CompTable ct,
                                                                const uint32_t* __restrict__ tile_pre,
                                                                uint32_t* __restrict__ comp_codes,
                                                                int16_t* __restrict__ res) {
    __shared__ int s_stream;
    __shared__ uint32_t s_part[DEC_THREADS / 32];
    __shared__ uint32_t s_ctok[DEC_MAX_COMP];
    __shared__ uint32_t s_cc[DEC_MAX_COMP];     // codes of the tile per component of its stream
    const int ntiles = (int)tile_base[nstreams];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
        const int s = dec_tile_stream(tile_base, nstreams, tile, &s_stream);
        const SDesc& D = sd[s];
        for (int i = threadIdx.x; i < D.ncomp; i += DEC_THREADS) {
            s_ctok[i] = comp_tok[D.comp0 + i];
            s_cc[i] = 0;
        }
        __syncthreads();
        const uint32_t ntok = rs[s].dec_tokens;
        const uint32_t t0 = (uint32_t)(tile - (int)tile_base[s]) * DEC_TILE + DEC_PER_THREAD * threadIdx.x;
        DecGroup G;
        uint32_t sum = 0;
        if (t0 < ntok) {
            G = dec_group(sc[s].in + D.hdr_bytes, t0, ntok, s_ctok, D.ncomp, D.comp0, rs[s].dec_type == 0, ct);
#pragma unroll
            for (int k = 0; k < DEC_PER_THREAD; k++) sum += G.n[k];
        }
        // block exclusive scan of the threads' codes
        uint32_t x = sum;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
            if (lane >= o) x += y;
        }
        if (lane == 31) s_part[warp] = x;
        __syncthreads();
        uint32_t wpre = 0;
#pragma unroll
        for (int i = 0; i < DEC_THREADS / 32; i++)
            if (i < warp) wpre += s_part[i];
        // codes per component: the group's first component's codes are summed over the
        // lanes sharing it (one shared-memory add per component per warp), the rest added alone
        int cfirst = -1;
        uint32_t cs_first = 0;
        if (t0 < ntok) {
            const int d = min((int)rs[s].dec_drop, CVC_MAX_LEVELS);
            const long long ndense = D.ncoef - absent_before(D, d, 3);
            long long p = (long long)(tile_pre[tile] - tile_pre[tile_base[s]]) + wpre + x - sum;
            cfirst = G.comp[0] - D.comp0;
            int cprev = cfirst;
            uint32_t csum = 0;
#pragma unroll
            for (int k = 0; k < DEC_PER_THREAD; k++) {
                if (G.comp[k] < 0) break;
                const int cl = G.comp[k] - D.comp0;
                if (cl != cprev) {
                    if (cprev == cfirst) cs_first = csum;
                    else if (csum) atomicAdd(&s_cc[cprev], csum);
                    cprev = cl;
                    csum = 0;
                }
                csum += G.n[k];
                if (G.code[k] && p >= 0 && p < ndense) res[D.coef_off + (d > 0 ? dense_to_layout(D, d, p) : p)] = G.v[k];
                p += G.n[k];
            }
            if (cprev == cfirst) cs_first = csum;
            else if (csum) atomicAdd(&s_cc[cprev], csum);
        }
        const unsigned peers = __match_any_sync(0xffffffffu, cfirst);
        const uint32_t tot = __reduce_add_sync(peers, cs_first);
        if (cfirst >= 0 && lane == __ffs(peers) - 1 && tot) atomicAdd(&s_cc[cfirst], tot);
        __syncthreads();
        for (int i = threadIdx.x; i < D.ncomp; i += DEC_THREADS)
            if (s_cc[i]) atomicAdd(&comp_codes[D.comp0 + i], s_cc[i]);
        __syncthreads();   // shared arrays are reused by the next tile
    }
}

// every component must expand to exactly its number of codes (none if dropped)
__global__ void k_dec_check_b(const SDesc* __restrict__ sd, const SResult* __restrict__ rs,
                              const uint32_t* __restrict__ comp_codes, CompTable ct, SResult* out) {
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= ct.ncomp) return;
    const int s = ct.stream[c];
    if (rs[s].dec_tokens == 0) return;        // not decoding, or the header was rejected
    const SDesc& D = sd[s];
    const int d = min((int)rs[s].dec_drop, CVC_MAX_LEVELS);
    const int lv = ct.level[c];
    const long long size = (c + 1 < D.comp0 + D.ncomp ? ct.elem[c + 1] : D.ncoef) - ct.elem[c];
    const long long want = (lv >= 1 && lv <= d) ? 0 : size;
    if ((long long)comp_codes[c] != want) atomicOr(&out[s].dec_err, EF_CORRUPT);
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

void launch_quant_b(bool pow2, int nblocks, cudaStream_t st, const float* coef, int16_t* est0, int16_t* est1,
                    const PDesc* pd, const int* blk_plane, const SDesc* sd, const SCall* sc, int16_t* res,
                    SResult* out) {
    if (pow2) k_quant_b<true><<<nblocks, ELEM_THREADS, 0, st>>>(coef, est0, est1, pd, blk_plane, sd, sc, res, out);
    else k_quant_b<false><<<nblocks, ELEM_THREADS, 0, st>>>(coef, est0, est1, pd, blk_plane, sd, sc, res, out);
}

}  // namespace cvc
