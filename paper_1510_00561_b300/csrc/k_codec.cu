// k_codec.cu -- the codec's element-wise and row-wise stages:
//   colour conversion + 4:2:0 + padding (§3.1), quantisation with lowpass
//   normalisation and thresholding (§3.4-§3.6), K/P differencing (§3.7),
//   run-length coding of rows (§3.8), their inverses, and a device-wide scan.
#include "k_codec.cuh"

namespace cvc {

__device__ __forceinline__ int mirror_idx(int a, int n) { return a < n ? a : 2 * n - 1 - a; }

// ------------------------------------------------------------- colour
// YCoCg-R lifting (integer form of Table 1): Co = R-B, t = B + (Co>>1),
// Cg = G - t, Y = t + (Cg>>1).  Luma items write the padded Y plane, chroma
// items the padded 2x2-averaged Co / Cg planes (rounded mean, odd edges
// replicated); padding mirrors about the last row / column.
__global__ void k_colour_fwd(const uint8_t* __restrict__ rgb, long long pitch, ColourGeom g, float* __restrict__ Y,
                             float* __restrict__ Co, float* __restrict__ Cg) {
    const long long nY = (long long)g.Hp * g.Wp, nC = (long long)g.Hcp * g.Wcp;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < nY + nC;
         i += (long long)gridDim.x * blockDim.x) {
        if (i < nY) {
            int y = (int)(i / g.Wp), x = (int)(i - (long long)y * g.Wp);
            int sy = mirror_idx(y, g.H), sx = mirror_idx(x, g.W);
            const uint8_t* p = rgb + sy * pitch + 3 * sx;
            int R = p[0], G = p[1], Bv = p[2];
            int co = R - Bv, t = Bv + (co >> 1), cg = G - t;
            Y[i] = (float)(t + (cg >> 1));
        } else {
            long long k = i - nY;
            int cy = (int)(k / g.Wcp), cx = (int)(k - (long long)cy * g.Wcp);
            int sy = mirror_idx(cy, g.Hc), sx = mirror_idx(cx, g.Wc);
            int r0 = 2 * sy, r1 = min(2 * sy + 1, g.H - 1), c0 = 2 * sx, c1 = min(2 * sx + 1, g.W - 1);
            int sco = 0, scg = 0;
            const int rr[2] = {r0, r1}, cc[2] = {c0, c1};
#pragma unroll
            for (int a = 0; a < 2; a++)
#pragma unroll
                for (int b = 0; b < 2; b++) {
                    const uint8_t* p = rgb + rr[a] * pitch + 3 * cc[b];
                    int R = p[0], G = p[1], Bv = p[2];
                    int co = R - Bv, t = Bv + (co >> 1);
                    sco += co;
                    scg += G - t;
                }
            Co[k] = (float)((sco + 2) >> 2);
            Cg[k] = (float)((scg + 2) >> 2);
        }
    }
}

__device__ __forceinline__ int round_clamp(float v, int lo, int hi) {
    float r = roundf(v);
    r = fminf(fmaxf(r, (float)lo), (float)hi);
    return (int)r;
}

// Decoder end: round (ties away from zero) and clamp the reconstructed
// planes, bilinear (9,3,3,1)/16 chroma upsampling with centred siting and
// clamped edges, inverse YCoCg-R, clamp to [0, 255].
__global__ void k_colour_inv(const float* __restrict__ Y, const float* __restrict__ Co, const float* __restrict__ Cg,
                             ColourGeom g, uint8_t* __restrict__ rgb, long long pitch) {
    const long long n = (long long)g.H * g.W;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        int y = (int)(i / g.W), x = (int)(i - (long long)y * g.W);
        int yy = round_clamp(Y[(long long)y * g.Wp + x], 0, 255);
        int i0 = min(y >> 1, g.Hc - 1), i1 = (y & 1) ? min((y >> 1) + 1, g.Hc - 1) : max((y >> 1) - 1, 0);
        int j0 = min(x >> 1, g.Wc - 1), j1 = (x & 1) ? min((x >> 1) + 1, g.Wc - 1) : max((x >> 1) - 1, 0);
        int c[2];
        const float* P[2] = {Co, Cg};
#pragma unroll
        for (int q = 0; q < 2; q++) {
            const float* p = P[q];
            int a = round_clamp(p[(long long)i0 * g.Wcp + j0], -255, 255);
            int b = round_clamp(p[(long long)i1 * g.Wcp + j0], -255, 255);
            int d = round_clamp(p[(long long)i0 * g.Wcp + j1], -255, 255);
            int e = round_clamp(p[(long long)i1 * g.Wcp + j1], -255, 255);
            c[q] = (9 * a + 3 * b + 3 * d + e + 8) >> 4;
        }
        int t = yy - (c[1] >> 1);
        int G = c[1] + t;
        int Bv = t - (c[0] >> 1);
        int R = Bv + c[0];
        uint8_t* o = rgb + y * pitch + 3 * x;
        o[0] = (uint8_t)min(max(R, 0), 255);
        o[1] = (uint8_t)min(max(G, 0), 255);
        o[2] = (uint8_t)min(max(Bv, 0), 255);
    }
}

// ------------------------------------------------------ quantisation + K/P
__device__ __forceinline__ int plane_of(const FrameGeom& f, long long e) {
    return e < f.poff[1] ? 0 : (e < f.poff[2] ? 1 : 2);
}

__device__ __forceinline__ int quant(float c, bool low, const QuantParams& q, uint32_t* err) {
    float t;
    if (low) t = c * q.low_scale;                    // exact power-of-two normalisation
    else t = (fabsf(c) >= q.threshold) ? c : 0.0f;
    float v = roundf(t / (low ? q.qpl : q.qph));     // IEEE division, ties away from zero
    if (!(fabsf(v) <= 32767.0f)) {
        atomicOr(err, EF_OVERFLOW);
        return 0;
    }
    return (int)v;
}

// codes q (the next coder state) and residuals r of one frame
__global__ void k_quant(const float* __restrict__ coef, const int16_t* __restrict__ prev, FrameGeom f, QuantParams qp,
                        int is_key, int16_t* __restrict__ q_out, int16_t* __restrict__ r_out, uint32_t* err) {
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < f.total;
         e += (long long)gridDim.x * blockDim.x) {
        int p = plane_of(f, e);
        long long le = e - f.poff[p];
        bool low = le < f.low_n[p];
        int q = quant(coef[e], low, qp, err);
        int r;
        if (!is_key) r = q - prev[e];
        else if (low && le >= f.low_w[p]) r = q - quant(coef[e - f.low_w[p]], true, qp, err);
        else r = q;
        q_out[e] = (int16_t)q;
        r_out[e] = (int16_t)(uint16_t)(r & 0xFFFF);   // wrapping 16-bit difference
    }
}

// decoder side: codes from residuals, then dequantised coefficients
__global__ void k_unquant(const int16_t* __restrict__ res, const int16_t* __restrict__ prev, FrameGeom f,
                          QuantParams qp, const DecInfo* __restrict__ info, int16_t* __restrict__ q_out,
                          float* __restrict__ coef) {
    const int is_key = info->type == 0;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < f.total;
         e += (long long)gridDim.x * blockDim.x) {
        int p = plane_of(f, e);
        long long le = e - f.poff[p];
        bool low = le < f.low_n[p];
        if (is_key && low) continue;                  // column prefix sums: k_unquant_keylow
        int q = is_key ? res[e] : (int16_t)(uint16_t)((res[e] + prev[e]) & 0xFFFF);
        q_out[e] = (int16_t)q;
        coef[e] = (float)q * (low ? qp.qpl_denorm : qp.qph);
    }
}

// K-frame lowpass: undo the column first difference (running sum down each column)
__global__ void k_unquant_keylow(const int16_t* __restrict__ res, FrameGeom f, QuantParams qp,
                                 const DecInfo* __restrict__ info, int16_t* __restrict__ q_out,
                                 float* __restrict__ coef) {
    if (info->type != 0) return;
    int t = blockIdx.x * blockDim.x + threadIdx.x;
    for (int p = 0; p < 3; p++) {
        if (t >= f.low_w[p]) { t -= f.low_w[p]; continue; }
        long long base = f.poff[p] + t;
        int rows = (int)(f.low_n[p] / f.low_w[p]);
        int acc = 0;
        for (int r = 0; r < rows; r++) {
            long long e = base + (long long)r * f.low_w[p];
            acc = (int16_t)(uint16_t)((acc + res[e]) & 0xFFFF);
            q_out[e] = (int16_t)acc;
            coef[e] = (float)acc * qp.qpl_denorm;
        }
        return;
    }
}

// ------------------------------------------------------------------ RLE
// Rows of every component, in stream order.  Token count of a row: one per
// non-zero code plus two per maximal zero run; raw rows (K-frame lowpass)
// carry one token per code.
__global__ void k_rle_count(const int16_t* __restrict__ res, const RowTable rt, int is_key, uint32_t* __restrict__ cnt) {
    const int lane = threadIdx.x & 31;
    const int row = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (row >= rt.nrows) return;
    const long long off = rt.off[row];
    const int w = rt.w[row];
    if (is_key && rt.low[row]) {
        if (lane == 0) cnt[row] = (uint32_t)w;
        return;
    }
    uint32_t n = 0;
    bool prev_zero = false;
    for (int x0 = 0; x0 < w; x0 += 32) {
        int x = x0 + lane;
        bool valid = x < w;
        bool z = valid && res[off + x] == 0;
        unsigned zb = __ballot_sync(0xffffffffu, z);
        unsigned vb = __ballot_sync(0xffffffffu, valid);
        unsigned prevz = (zb << 1) | (prev_zero ? 1u : 0u);
        unsigned starts = zb & ~prevz;
        n += __popc(vb & ~zb) + 2 * __popc(starts);
        prev_zero = (zb >> 31) & 1u;
    }
    if (lane == 0) cnt[row] = n;
}

__device__ __forceinline__ void put_tok(uint8_t* tok_base, uint32_t pos, uint32_t cap_tok, int16_t v, uint32_t* err) {
    if (pos < cap_tok) reinterpret_cast<int16_t*>(tok_base)[pos] = v;
    else atomicOr(err, EF_CAPACITY);
}

__global__ void k_rle_write(const int16_t* __restrict__ res, const RowTable rt, int is_key,
                            const uint32_t* __restrict__ tokoff, uint8_t* __restrict__ tok_base, uint32_t cap_tok,
                            uint32_t* err) {
    const int lane = threadIdx.x & 31;
    const int row = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (row >= rt.nrows) return;
    const long long off = rt.off[row];
    const int w = rt.w[row];
    uint32_t pos = tokoff[row];
    if (is_key && rt.low[row]) {
        for (int x = lane; x < w; x += 32) put_tok(tok_base, pos + x, cap_tok, res[off + x], err);
        return;
    }
    const unsigned lt = (1u << lane) - 1u;
    bool prev_zero = false;
    uint32_t open_pos = 0;   // token position of the marker of a run left open by the previous chunk
    int open_x = 0;
    for (int x0 = 0; x0 < w; x0 += 32) {
        int x = x0 + lane;
        bool valid = x < w;
        int16_t v = valid ? res[off + x] : (int16_t)1;
        bool z = valid && v == 0;
        unsigned zb = __ballot_sync(0xffffffffu, z);
        unsigned vb = __ballot_sync(0xffffffffu, valid);
        unsigned starts = zb & ~((zb << 1) | (prev_zero ? 1u : 0u));
        unsigned nz = vb & ~zb;
        bool start = (starts >> lane) & 1u;
        uint32_t my = pos + __popc(nz & lt) + 2 * __popc(starts & lt);
        if (valid && !z) put_tok(tok_base, my, cap_tok, v, err);
        if (start) put_tok(tok_base, my, cap_tok, 0, err);
        // the run containing this lane started at the highest start lane <= lane, or before the chunk
        unsigned le = starts & (lt | (1u << lane));
        int sl = le ? 31 - __clz(le) : -1;
        uint32_t spos = __shfl_sync(0xffffffffu, my, sl < 0 ? 0 : sl);
        int sx = sl < 0 ? open_x : x0 + sl;
        if (sl < 0) spos = open_pos;
        // this lane ends its run if it is zero and the next element is not (or the row ends)
        bool next_zero;
        if (lane < 31) next_zero = (zb >> (lane + 1)) & 1u;
        else next_zero = (x + 1 < w) && res[off + x + 1] == 0;
        if (z && !next_zero) put_tok(tok_base, spos + 1, cap_tok, (int16_t)(x - sx + 1), err);
        // carry an open run into the next chunk
        int src31 = 31;
        uint32_t spos31 = __shfl_sync(0xffffffffu, spos, src31);
        int sx31 = __shfl_sync(0xffffffffu, sx, src31);
        prev_zero = (zb >> 31) & 1u;
        if (prev_zero) {
            open_pos = spos31;
            open_x = sx31;
        }
        pos += __popc(nz) + 2 * __popc(starts);
    }
}

__global__ void k_stream_header(StreamHeader h, const uint32_t* __restrict__ tokoff, const int* __restrict__ comp_row0,
                                int ncomp, uint8_t* __restrict__ out, uint32_t* __restrict__ info) {
    int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t == 0) {
        uint8_t* o = out;
        o[0] = 'C'; o[1] = 'V'; o[2] = 'C'; o[3] = '1';
        o[4] = 1; o[5] = 0;
        o[6] = (uint8_t)h.type;
        o[7] = (uint8_t)h.levels;
        for (int i = 0; i < 4; i++) o[8 + i] = (uint8_t)(h.frame_index >> (8 * i));
        o[12] = (uint8_t)h.height; o[13] = (uint8_t)(h.height >> 8);
        o[14] = (uint8_t)h.width; o[15] = (uint8_t)(h.width >> 8);
        for (int i = 0; i < 6; i++) o[16 + i] = (uint8_t)h.dirs[i];
        o[22] = (uint8_t)h.qph; o[23] = (uint8_t)(h.qph >> 8);
        o[24] = (uint8_t)h.qpl; o[25] = (uint8_t)(h.qpl >> 8);
        o[26] = 0; o[27] = 0;
        for (int i = 0; i < 4; i++) o[28 + i] = (uint8_t)((unsigned)ncomp >> (8 * i));
        info[0] = tokoff[comp_row0[ncomp]];
    }
    if (t < ncomp) {
        uint32_t c = tokoff[comp_row0[t + 1]] - tokoff[comp_row0[t]];
        reinterpret_cast<uint32_t*>(out + 32)[t] = c;
    }
}

// ------------------------------------------------------------ decoding
__device__ __forceinline__ uint32_t rd32(const uint8_t* p) {
    return (uint32_t)p[0] | ((uint32_t)p[1] << 8) | ((uint32_t)p[2] << 16) | ((uint32_t)p[3] << 24);
}
__device__ __forceinline__ int16_t rd16(const uint8_t* p) { return (int16_t)(uint16_t)(p[0] | (p[1] << 8)); }

// header check, component token offsets (single block)
__global__ void k_dec_parse(const uint8_t* __restrict__ in, long long in_len, StreamHeader expect, int ncomp,
                            long long expect_next, uint32_t max_tok, uint32_t* __restrict__ comp_tok,
                            DecInfo* __restrict__ info, uint32_t* err) {
    __shared__ uint32_t s_carry;
    __shared__ int s_bad;
    __shared__ uint32_t s_part[1024];
    if (threadIdx.x == 0) {
        int bad = 0;
        info->type = 0;
        info->total = 0;
        if (in_len < 32 + 4LL * ncomp) bad = EF_CORRUPT;
        else {
            if (in[0] != 'C' || in[1] != 'V' || in[2] != 'C' || in[3] != '1' || in[4] != 1 || in[5] != 0) bad = EF_CORRUPT;
            int type = in[6];
            if (type > 1) bad = EF_CORRUPT;
            if (in[7] != expect.levels || (in[12] | (in[13] << 8)) != expect.height ||
                (in[14] | (in[15] << 8)) != expect.width || (in[22] | (in[23] << 8)) != expect.qph ||
                (in[24] | (in[25] << 8)) != expect.qpl || rd32(in + 28) != (uint32_t)ncomp)
                bad |= EF_MISMATCH;
            for (int i = 0; i < 6; i++)
                if (in[16 + i] != expect.dirs[i]) bad |= EF_MISMATCH;
            uint32_t fidx = rd32(in + 8);
            if (!bad && type == 1 && (expect_next < 0 || (long long)fidx != expect_next)) bad |= EF_STATE;
            info->type = type;
            info->frame_index = fidx;
        }
        s_bad = bad;
        s_carry = 0;
    }
    __syncthreads();
    if (s_bad) {
        if (threadIdx.x == 0) atomicOr(err, (uint32_t)s_bad);
        return;
    }
    // exclusive scan of the ncomp token counts
    for (int base = 0; base < ncomp; base += blockDim.x) {
        int i = base + threadIdx.x;
        uint32_t v = i < ncomp ? rd32(in + 32 + 4 * i) : 0;
        s_part[threadIdx.x] = v;
        __syncthreads();
        for (int d = 1; d < (int)blockDim.x; d <<= 1) {
            uint32_t a = threadIdx.x >= (unsigned)d ? s_part[threadIdx.x - d] : 0;
            __syncthreads();
            s_part[threadIdx.x] += a;
            __syncthreads();
        }
        if (i < ncomp) comp_tok[i] = s_carry + s_part[threadIdx.x] - v;
        __syncthreads();
        if (threadIdx.x == blockDim.x - 1) s_carry += s_part[threadIdx.x];
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        uint32_t total = s_carry;
        comp_tok[ncomp] = total;
        if (32 + 4LL * ncomp + 2LL * total > in_len || total > max_tok) {
            atomicOr(err, EF_CORRUPT);
            total = 0;
        }
        info->total = total;
    }
}

__device__ __forceinline__ int find_comp(const uint32_t* comp_tok, int ncomp, uint32_t t) {
    int lo = 0, hi = ncomp - 1;  // largest c with comp_tok[c] <= t
    while (lo < hi) {
        int mid = (lo + hi + 1) >> 1;
        if (comp_tok[mid] <= t) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

// elements produced by each token: value (and raw K-lowpass) tokens 1,
// zero markers 0, run counts n.
__global__ void k_dec_contrib(const uint8_t* __restrict__ tok, const uint32_t* __restrict__ comp_tok, int ncomp,
                              const uint8_t* __restrict__ comp_low, const DecInfo* __restrict__ info,
                              uint32_t* __restrict__ contrib, uint32_t max_tok, uint32_t* err) {
    const uint32_t total = info->total;
    const int is_key = info->type == 0;
    for (uint32_t t = blockIdx.x * blockDim.x + threadIdx.x; t < max_tok; t += gridDim.x * blockDim.x) {
        if (t >= total) {
            contrib[t] = 0;
            continue;
        }
        int c = find_comp(comp_tok, ncomp, t);
        uint32_t c0 = comp_tok[c], c1 = comp_tok[c + 1];
        int16_t v = rd16(tok + 2LL * t);
        uint32_t n;
        if (is_key && comp_low[c]) n = 1;
        else if (t > c0 && rd16(tok + 2LL * (t - 1)) == 0) {
            n = v > 0 ? (uint32_t)v : 0;
            if (v <= 0) atomicOr(err, EF_CORRUPT);
        } else if (v != 0) n = 1;
        else {
            n = 0;
            if (t + 1 >= c1) atomicOr(err, EF_CORRUPT);
        }
        contrib[t] = n;
    }
}

// every component must expand to exactly its number of codes
__global__ void k_dec_check(const uint32_t* __restrict__ comp_tok, const uint32_t* __restrict__ pos,
                            const long long* __restrict__ comp_elem, int ncomp, const DecInfo* __restrict__ info,
                            uint32_t* err) {
    int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c > ncomp || info->total == 0) return;
    if ((long long)pos[comp_tok[c]] != comp_elem[c]) atomicOr(err, EF_CORRUPT);
}

__global__ void k_dec_scatter(const uint8_t* __restrict__ tok, const uint32_t* __restrict__ comp_tok, int ncomp,
                              const uint8_t* __restrict__ comp_low, const DecInfo* __restrict__ info,
                              const uint32_t* __restrict__ pos, long long ncoef, int16_t* __restrict__ res) {
    const uint32_t total = info->total;
    const int is_key = info->type == 0;
    for (uint32_t t = blockIdx.x * blockDim.x + threadIdx.x; t < total; t += gridDim.x * blockDim.x) {
        int16_t v = rd16(tok + 2LL * t);
        int c = find_comp(comp_tok, ncomp, t);
        bool raw = is_key && comp_low[c];
        bool count = !raw && t > comp_tok[c] && rd16(tok + 2LL * (t - 1)) == 0;
        if ((raw || (v != 0 && !count)) && (long long)pos[t] < ncoef) res[pos[t]] = v;
    }
}

// ------------------------------------------------------ exclusive scan
constexpr int SCAN_CHUNK = 2048;

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

__global__ void k_scan_reduce(const uint32_t* __restrict__ in, uint32_t n, uint32_t* __restrict__ sums) {
    __shared__ uint32_t sh[32];
    uint32_t base = blockIdx.x * SCAN_CHUNK, v = 0;
    for (uint32_t i = base + threadIdx.x; i < min(base + SCAN_CHUNK, n); i += blockDim.x) v += in[i];
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

__global__ void k_scan_apply(const uint32_t* __restrict__ in, uint32_t n, const uint32_t* __restrict__ sums,
                             uint32_t* __restrict__ out) {
    __shared__ uint32_t wsum[32];
    uint32_t base = blockIdx.x * SCAN_CHUNK;
    // each thread owns SCAN_CHUNK / blockDim consecutive elements
    const int per = SCAN_CHUNK / blockDim.x;
    uint32_t loc[16];
    uint32_t tsum = 0;
    for (int k = 0; k < per; k++) {
        uint32_t i = base + threadIdx.x * per + k;
        loc[k] = i < n ? in[i] : 0;
        tsum += loc[k];
    }
    // block exclusive scan of thread sums
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
    uint32_t excl = x - tsum + ((threadIdx.x >> 5) ? wsum[(threadIdx.x >> 5) - 1] : 0) + sums[blockIdx.x];
    for (int k = 0; k < per; k++) {
        uint32_t i = base + threadIdx.x * per + k;
        if (i < n) out[i] = excl;
        excl += loc[k];
    }
    if (blockIdx.x == gridDim.x - 1 && threadIdx.x == 0) out[n] = sums[gridDim.x];
}

cudaError_t exclusive_scan(const uint32_t* in, uint32_t n, uint32_t* out, uint32_t* tmp, cudaStream_t st) {
    int nb = (int)((n + SCAN_CHUNK - 1) / SCAN_CHUNK);
    if (nb == 0) nb = 1;
    k_scan_reduce<<<nb, 256, 0, st>>>(in, n, tmp);
    k_scan_sums<<<1, 1024, 0, st>>>(tmp, nb);
    k_scan_apply<<<nb, 256, 0, st>>>(in, n, tmp, out);
    return cudaGetLastError();   // three launches, counted by the caller
}

}  // namespace cvc
