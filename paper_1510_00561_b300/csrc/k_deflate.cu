// k_deflate.cu -- the DEFLATE stage of CVC (§3.9).  Scalable mode: every
// component's token bytes become one raw DEFLATE stream (RFC 1951) of its
// own, so that a receiver can be sent any subset of components.  CVC-NTS
// mode: the token bytes of the whole frame become one stream.
//
// Each stream is one final block with dynamic Huffman codes over literal
// bytes only (the Huffman-only strategy: no LZ77 matches), which makes both
// directions data-parallel:
//   deflate  a byte histogram per stream, one length-limited Huffman code
//            per stream (a block each), the block header, and the data
//            written by one thread per 256-byte segment at a bit offset from
//            a scan of the segments' bit lengths;
//   inflate  a block per stream decodes its block header into decoding
//            tables, one thread per segment decodes its 256 literals
//            starting at the bit offset the container records.
// Segments are handled in groups of 256 (a block each), so that one large
// stream spreads over many blocks.
// The container keeps the CVC header and token counts, adds each stream's
// byte length and the bit length of each of its segments (the entry points
// of the parallel inflate), then the streams, then the motion vectors.  Any
// inflater reads every stream on its own; the segment table only lets the
// GPU start in the middle.
#include <algorithm>
#include <cstring>

#include "k_deflate.cuh"

namespace cvc {

namespace {

__device__ __forceinline__ uint32_t rd32(const uint8_t* p) {
    return (uint32_t)p[0] | ((uint32_t)p[1] << 8) | ((uint32_t)p[2] << 16) | ((uint32_t)p[3] << 24);
}
__device__ __forceinline__ void wr32(uint8_t* p, uint32_t v) {
    p[0] = (uint8_t)v; p[1] = (uint8_t)(v >> 8); p[2] = (uint8_t)(v >> 16); p[3] = (uint8_t)(v >> 24);
}
__device__ __forceinline__ uint32_t bit_reverse(uint32_t code, int len) { return __brev(code) >> (32 - len); }

// the order in which the code-length code's lengths are sent (RFC 1951, 3.2.7)
__constant__ uint8_t CL_ORDER[19] = {16, 17, 18, 0, 8, 7, 9, 6, 10, 5, 11, 4, 12, 3, 13, 2, 14, 1, 15};

// canonical codes (RFC 1951, 3.2.2), bit-reversed for LSB-first emission
__device__ void canonical_codes(const uint8_t* len, int n, uint16_t* code) {
    uint16_t count[16] = {0}, next[16];
    for (int i = 0; i < n; i++) count[len[i]]++;
    count[0] = 0;
    uint16_t c = 0;
    for (int b = 1; b < 16; b++) {
        c = (uint16_t)((c + count[b - 1]) << 1);
        next[b] = c;
    }
    for (int i = 0; i < n; i++)
        code[i] = len[i] ? (uint16_t)bit_reverse(next[len[i]]++, len[i]) : 0;
}

// sequential bit writer into a byte buffer (zeroed by the caller)
struct BitOut {
    uint8_t* p;
    uint32_t pos, cap;     // bits written, bit capacity
    bool over;
    unsigned long long acc = 0;   // the nacc bits after the last stored byte
    int nacc = 0;
    __device__ void put(uint32_t v, int n) {
        if (pos + n > cap) { over = true; return; }
        acc |= (unsigned long long)(v & ((n < 32) ? ((1u << n) - 1u) : 0xFFFFFFFFu)) << nacc;
        nacc += n;
        pos += n;
        while (nacc >= 8) {
            p[(pos - nacc) >> 3] = (uint8_t)acc;
            acc >>= 8;
            nacc -= 8;
        }
    }
    __device__ void flush() {
        if (nacc > 0) p[(pos - nacc) >> 3] = (uint8_t)acc;
        acc = 0;
        nacc = 0;
    }
};

// canonical decoding arrays of a code: codes per length, symbols in code order.
// Kept out of line: inlined into k_ifl_tables with its local tables, our
// sm_103a build decoded wrong symbols, while the same source run on the host
// and the out-of-line form are correct.
__device__ __noinline__ bool build_decoder(const uint8_t* len, int n, uint16_t* count, uint16_t* sym) {
    for (int b = 0; b < 16; b++) count[b] = 0;
    for (int i = 0; i < n; i++) count[len[i]]++;
    count[0] = 0;
    // over-subscribed codes are invalid (an incomplete code is allowed, as in RFC 1951 inflaters)
    int left = 1;
    for (int b = 1; b < 16; b++) {
        left <<= 1;
        left -= count[b];
        if (left < 0) return false;
    }
    uint16_t offs[16];
    offs[1] = 0;
    for (int b = 1; b < 15; b++) offs[b + 1] = (uint16_t)(offs[b] + count[b]);
    for (int i = 0; i < n; i++)
        if (len[i]) sym[offs[len[i]]++] = (uint16_t)i;
    return true;
}

// exclusive scan of one value per thread over a block of 256 threads; *total = the sum
__device__ unsigned long long block_scan(unsigned long long v, unsigned long long* sh, unsigned long long* total) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    unsigned long long x = v;
    for (int o = 1; o < 32; o <<= 1) {
        const unsigned long long y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) sh[warp] = x;
    __syncthreads();
    if (warp == 0) {
        unsigned long long t = lane < 8 ? sh[lane] : 0;
        for (int o = 1; o < 8; o <<= 1) {
            const unsigned long long y = __shfl_up_sync(0xffffffffu, t, o);
            if (lane >= o) t += y;
        }
        if (lane < 8) sh[lane] = t;
    }
    __syncthreads();
    const unsigned long long r = (warp ? sh[warp - 1] : 0) + x - v;
    *total = sh[7];
    __syncthreads();
    return r;
}

// Huffman lengths of the (at most 19) code-length symbols, limited to maxlen:
// leaves sorted by (weight, symbol), two queues, halving the weights while too deep
__device__ void small_huffman(const uint32_t* f, int n, int maxlen, uint8_t* len) {
    uint32_t w[40];
    uint8_t ord[20], q[20], parent[40];
    for (int i = 0; i < n; i++) w[i] = f[i];
    for (;;) {
        int nu = 0;
        for (int i = 0; i < n; i++) {
            len[i] = 0;
            if (!w[i]) continue;
            int k = nu++;
            while (k > 0 && (w[ord[k - 1]] > w[i])) { ord[k] = ord[k - 1]; k--; }
            ord[k] = (uint8_t)i;
        }
        if (nu < 2) {                      // a lone symbol: one bit (the caller completes the code)
            for (int i = 0; i < n; i++) len[i] = w[i] ? 1 : 0;
            return;
        }
        int li = 0, qh = 0, qt = 0, m = n;
        auto take = [&]() -> int {
            if (li < nu && (qh >= qt || w[ord[li]] <= w[q[qh]])) return ord[li++];
            return q[qh++];
        };
        for (int k = 0; k < nu - 1; k++) {
            const int x = take(), y = take();
            w[m] = w[x] + w[y];
            parent[x] = parent[y] = (uint8_t)m;
            q[qt++] = (uint8_t)m;
            m++;
        }
        const int root = m - 1;
        int deep = 0;
        for (int i = 0; i < n; i++) {
            if (!w[i]) continue;
            int d = 0;
            for (int x = i; x != root; x = parent[x]) d++;
            len[i] = (uint8_t)d;
            deep = max(deep, d);
        }
        if (deep <= maxlen) return;
        for (int i = 0; i < n; i++) w[i] = w[i] ? (w[i] + 1) >> 1 : 0;
    }
}

// the stream of group g: the last stream whose first group is <= g
__device__ __forceinline__ int group_stream(const DflComp* comp, int nstr, uint32_t g) {
    int lo = 0, hi = nstr;
    while (hi - lo > 1) {
        const int mid = (lo + hi) >> 1;
        if (comp[mid].grp0 <= g) lo = mid;
        else hi = mid;
    }
    while (lo + 1 < nstr && comp[lo + 1].grp0 <= g) lo++;
    return lo;
}

}  // namespace

// -------------------------------------------------------------- deflate
// stream byte offsets of the input tokens, segments, groups (one block per frame)
__global__ void __launch_bounds__(256) k_dfl_plan(DflArgs a) {
    const DflFrame& F = a.fr[blockIdx.y];
    DflScratch& S = *F.S;
    __shared__ unsigned long long sh[8];
    __shared__ int s_bad;
    const uint8_t* in = F.in;
    if (threadIdx.x == 0) {
        S.err = 0;
        S.total = 0;
        s_bad = F.in_len < (long long)a.hdr_bytes || rd32(in) != 0x31435643u || in[4] != 1 || in[5] > 5 ||
                rd32(in + 28) != (uint32_t)a.ncomp;
        if (s_bad) S.err = DFL_CORRUPT;
    }
    __syncthreads();
    if (s_bad) return;
    const int nstr = a.nts ? 1 : a.ncomp;
    unsigned long long tok = 0, seg = 0, grp = 0, tt, ts, tg;
    for (int b = 0; b < a.ncomp; b += blockDim.x) {
        const int c = b + threadIdx.x;
        const uint32_t n = c < a.ncomp ? rd32(in + 32 + 4 * c) : 0;
        const unsigned long long segs = a.nts ? 0 : (2ULL * n + DFL_SEG - 1) / DFL_SEG;
        const unsigned long long grps = (segs + DFL_GRP - 1) / DFL_GRP;
        const unsigned long long pt = block_scan(n, sh, &tt), ps = block_scan(segs, sh, &ts),
                                 pg = block_scan(grps, sh, &tg);
        if (c < a.ncomp && !a.nts) {
            S.comp[c].in_off = a.hdr_bytes + 2 * (tok + pt);
            S.comp[c].bytes = 2ULL * n;
            S.comp[c].seg0 = (uint32_t)(seg + ps);
            S.comp[c].grp0 = (uint32_t)(grp + pg);
        }
        tok += tt;
        seg += ts;
        grp += tg;
    }
    if (a.nts) {                           // one stream over the frame's token bytes
        seg = (2 * tok + DFL_SEG - 1) / DFL_SEG;
        grp = (seg + DFL_GRP - 1) / DFL_GRP;
        if (threadIdx.x == 0) {
            S.comp[0].in_off = a.hdr_bytes;
            S.comp[0].bytes = 2 * tok;
            S.comp[0].seg0 = 0;
            S.comp[0].grp0 = 0;
        }
    }
    for (int i = threadIdx.x; i < nstr * DFL_NLIT; i += blockDim.x)
        S.hist[i] = (i % DFL_NLIT) == 256 ? 1u : 0u;      // the end-of-block code occurs once
    if (threadIdx.x == 0) {
        S.comp[nstr].seg0 = (uint32_t)seg;
        S.comp[nstr].grp0 = (uint32_t)grp;
        const int type = in[6];
        const long long mvb = type == 2 ? a.mv_bytes : 0;
        if ((type == 2 && a.mv_bytes == 0) || seg > (unsigned long long)a.max_seg ||
            grp > (unsigned long long)a.max_grp || a.hdr_bytes + 2 * tok + mvb > (unsigned long long)F.in_len) {
            S.err = DFL_CORRUPT;
            return;
        }
        S.nseg = (uint32_t)seg;
        S.nstr = (uint32_t)nstr;
        S.ngrp = (uint32_t)grp;
        S.tok_bytes = 2 * tok;
        S.tail = mvb;
    }
}

// byte histogram of each stream: one block per group of segments, a
// sub-histogram per warp in shared memory, added to the stream's
__global__ void __launch_bounds__(256) k_dfl_hist(DflArgs a) {
    const DflFrame& F = a.fr[blockIdx.y];
    DflScratch& S = *F.S;
    const uint32_t g = blockIdx.x;
    if (S.err || g >= S.ngrp) return;
    const int c = group_stream(S.comp, (int)S.nstr, g);
    const DflComp& C = S.comp[c];
    __shared__ uint32_t h[8][256];     // one per warp: the few common bytes collide less
    for (int i = threadIdx.x; i < 8 * 256; i += blockDim.x) h[i >> 8][i & 255] = 0;
    __syncthreads();
    const unsigned long long b0 = (unsigned long long)(g - C.grp0) * DFL_GRP * DFL_SEG;
    const unsigned long long b1 = min(C.bytes, b0 + (unsigned long long)DFL_GRP * DFL_SEG);
    const uint8_t* p = F.in + C.in_off;
    uint32_t* hw = h[(threadIdx.x >> 5) & 7];
    for (unsigned long long i = b0 + threadIdx.x; i < b1; i += blockDim.x) atomicAdd(&hw[p[i]], 1u);
    __syncthreads();
    for (int i = threadIdx.x; i < 256; i += blockDim.x) {
        uint32_t t = 0;
        for (int k = 0; k < 8; k++) t += h[k][i];
        if (t) atomicAdd(&S.hist[c * DFL_NLIT + i], t);
    }
}

// code of each stream (one block each): literal/length code lengths (two
// queues over the leaves sorted by (weight, symbol), in shared memory; the
// weights halved while a code would be longer than 15 bits), canonical codes,
// the run-length coded block header and its bit length
__global__ void __launch_bounds__(256) k_dfl_code(DflArgs a) {
    const DflFrame& F = a.fr[blockIdx.y];
    DflScratch& S = *F.S;
    const int c = blockIdx.x, tid = threadIdx.x;
    if (S.err || c >= (int)S.nstr) return;
    DflComp& C = S.comp[c];
    if (C.bytes == 0) {
        if (tid == 0) C.hdr_bits = 0, C.data_bits = 0;
        return;
    }
    __shared__ uint32_t w[2 * DFL_NLIT];
    __shared__ uint16_t parent[2 * DFL_NLIT], order[DFL_NLIT], q[DFL_NLIT], scode[DFL_NLIT];
    __shared__ uint8_t len[DFL_NLIT];
    __shared__ int s_n, s_root, s_deep, s_fixed;
    __shared__ uint16_t nextc[16];
    __shared__ uint8_t hbuf[DFL_HDR_BYTES];
    __shared__ unsigned long long sh[8];
    const uint32_t* hist = S.hist + c * DFL_NLIT;
    for (int i = tid; i < DFL_NLIT; i += blockDim.x) w[i] = hist[i];
    for (int round = 0; round < 40; round++) {
        if (tid == 0) s_n = 0, s_deep = 0;
        __syncthreads();
        // rank of each used leaf by (weight, symbol)
        for (int i = tid; i < DFL_NLIT; i += blockDim.x) {
            if (!w[i]) continue;
            int r = 0;
            for (int j = 0; j < DFL_NLIT; j++) r += w[j] && (w[j] < w[i] || (w[j] == w[i] && j < i));
            order[r] = (uint16_t)i;
            atomicAdd(&s_n, 1);
        }
        __syncthreads();
        if (tid == 0) {
            const int n = s_n;
            int li = 0, qh = 0, qt = 0, m = DFL_NLIT;
            for (int k = 0; k < n - 1; k++) {
                int x[2];
                for (int e = 0; e < 2; e++) {
                    if (li < n && (qh >= qt || w[order[li]] <= w[q[qh]])) x[e] = order[li++];
                    else x[e] = q[qh++];
                }
                w[m] = w[x[0]] + w[x[1]];
                parent[x[0]] = parent[x[1]] = (uint16_t)m;
                q[qt++] = (uint16_t)m;
                m++;
            }
            s_root = m - 1;
        }
        __syncthreads();
        for (int i = tid; i < DFL_NLIT; i += blockDim.x) {
            int d = 0;
            if (hist[i]) {
                for (int x = i; x != s_root; x = parent[x]) d++;
            }
            len[i] = (uint8_t)d;
            atomicMax(&s_deep, d);
        }
        __syncthreads();
        if (s_deep <= 15) break;
        if (round == 0) {
            // too deep: clamp to 15 bits and rebalance Kraft's sum by moving leaves one
            // level down from the deepest level below 15 (the overflow repair of zlib's
            // trees.c); the least frequent leaves then take the longest lengths
            if (tid == 0) {
                int cnt[16] = {0}, overflow = 0;
                for (int i = 0; i < DFL_NLIT; i++) {
                    if (!hist[i]) continue;
                    if (len[i] > 15) overflow++;
                    cnt[min((int)len[i], 15)]++;
                }
                while (overflow > 0) {
                    int b = 14;
                    while (b > 0 && cnt[b] == 0) b--;
                    if (b == 0) break;
                    cnt[b]--;
                    cnt[b + 1] += 2;
                    cnt[15]--;
                    overflow -= 2;
                }
                long long kraft = 0;
                for (int b = 1; b <= 15; b++) kraft += (long long)cnt[b] << (15 - b);
                int k = 0;
                for (int b = 15; b >= 1; b--)
                    for (int m = cnt[b]; m > 0; m--) len[order[k++]] = (uint8_t)b;
                // a flag of its own: other warps may still be reading s_deep above
                s_fixed = kraft == (1LL << 15) && k == s_n;
            }
            __syncthreads();
            if (s_fixed) break;
        }
        for (int i = tid; i < DFL_NLIT; i += blockDim.x) w[i] = w[i] ? (w[i] + 1) >> 1 : 0;
        __syncthreads();
    }
    // canonical codes (RFC 1951, 3.2.2): the codes of one length are consecutive in symbol order
    if (tid == 0) {
        uint16_t cnt[16] = {0};
        for (int i = 0; i < DFL_NLIT; i++) cnt[len[i]]++;
        cnt[0] = 0;
        uint16_t cc = 0;
        for (int b = 1; b < 16; b++) {
            cc = (uint16_t)((cc + cnt[b - 1]) << 1);
            nextc[b] = cc;
        }
    }
    __syncthreads();
    unsigned long long bits = 0;
    for (int i = tid; i < DFL_NLIT; i += blockDim.x) {
        const int l = len[i];
        uint16_t v = 0;
        if (l) {
            int r = 0;
            for (int j = 0; j < i; j++) r += len[j] == l;
            v = (uint16_t)bit_reverse(nextc[l] + r, l);
        }
        scode[i] = v;
        S.code[c * DFL_NLIT + i] = v;
        S.len[c * DFL_NLIT + i] = (uint8_t)l;
        bits += (unsigned long long)hist[i] * l;
    }
    unsigned long long total_bits;
    block_scan(bits, sh, &total_bits);
    // the block header (one thread): code lengths of the 257 literal/length codes and
    // two unused one-bit distance codes, run-length coded with the code-length alphabet
    if (tid == 0) {
        uint8_t rs[DFL_NLIT + 2], rx[DFL_NLIT + 2];
        const int N = DFL_NLIT + 2;
        auto seq = [&](int k) -> int { return k < DFL_NLIT ? len[k] : 1; };
        int nr = 0;
        for (int i = 0; i < N;) {
            const int v = seq(i);
            int run = 1;
            while (i + run < N && seq(i + run) == v) run++;
            if (v == 0) {
                int r = run;
                while (r >= 11) {
                    const int k = min(r, 138);
                    rs[nr] = 18; rx[nr++] = (uint8_t)(k - 11);
                    r -= k;
                }
                if (r >= 3) {
                    rs[nr] = 17; rx[nr++] = (uint8_t)(r - 3);
                    r = 0;
                }
                while (r-- > 0) { rs[nr] = 0; rx[nr++] = 0; }
            } else {
                rs[nr] = (uint8_t)v; rx[nr++] = 0;
                int r = run - 1;
                while (r >= 3) {
                    const int k = min(r, 6);
                    rs[nr] = 16; rx[nr++] = (uint8_t)(k - 3);
                    r -= k;
                }
                while (r-- > 0) { rs[nr] = (uint8_t)v; rx[nr++] = 0; }
            }
            i += run;
        }
        uint32_t cf[19] = {0};
        for (int i = 0; i < nr; i++) cf[rs[i]]++;
        uint8_t cl[19];
        uint16_t cc[19];
        small_huffman(cf, 19, 7, cl);
        int used = 0, only = 0;
        for (int i = 0; i < 19; i++)
            if (cf[i]) { used++; only = i; }
        if (used == 1) {
            cl[only] = 1;
            cl[only == 0 ? 1 : 0] = 1;
        }
        canonical_codes(cl, 19, cc);
        int hclen = 19;
        while (hclen > 4 && cl[CL_ORDER[hclen - 1]] == 0) hclen--;
        for (int i = 0; i < DFL_HDR_BYTES; i++) hbuf[i] = 0;
        BitOut o{hbuf, 0, DFL_HDR_BYTES * 8, false};
        o.put(1, 1);                   // BFINAL
        o.put(2, 2);                   // BTYPE = dynamic Huffman
        o.put(DFL_NLIT - 257, 5);      // HLIT
        o.put(1, 5);                   // HDIST: two distance codes
        o.put(hclen - 4, 4);           // HCLEN
        for (int i = 0; i < hclen; i++) o.put(cl[CL_ORDER[i]], 3);
        for (int i = 0; i < nr; i++) {
            o.put(cc[rs[i]], cl[rs[i]]);
            if (rs[i] == 16) o.put(rx[i], 2);
            else if (rs[i] == 17) o.put(rx[i], 3);
            else if (rs[i] == 18) o.put(rx[i], 7);
        }
        o.flush();
        if (o.over) S.err = DFL_INTERNAL;
        C.hdr_bits = o.pos;
        C.data_bits = total_bits;      // the literals and the end-of-block code
    }
    __syncthreads();
    uint8_t* hb = S.hdr + (size_t)c * DFL_HDR_BYTES;
    for (int i = tid; i < DFL_HDR_BYTES; i += blockDim.x) hb[i] = hbuf[i];
}

// stream offsets, container layout, the size check (one block)
__global__ void __launch_bounds__(256) k_dfl_layout(DflArgs a) {
    const DflFrame& F = a.fr[blockIdx.y];
    DflScratch& S = *F.S;
    __shared__ unsigned long long sh[8];
    if (S.err) return;
    const int nstr = (int)S.nstr;
    const unsigned long long tables = a.hdr_bytes + 4ULL * nstr + ((2ULL * S.nseg + 3) & ~3ULL);
    unsigned long long off = tables, tt;
    for (int b = 0; b < nstr; b += blockDim.x) {
        const int c = b + threadIdx.x;
        unsigned long long nb = 0;
        if (c < nstr) {
            const DflComp& C = S.comp[c];
            nb = C.bytes ? (C.hdr_bits + C.data_bits + 7) >> 3 : 0;
        }
        const unsigned long long p = block_scan(nb, sh, &tt);
        if (c < nstr) {
            S.comp[c].out_off = off + p;
            S.comp[c].out_bytes = nb;
        }
        off += tt;
    }
    if (threadIdx.x == 0) {
        S.streams = tables;
        S.total = off + S.tail;
        if (S.total > (unsigned long long)F.out_cap) S.err = DFL_CAPACITY;
    }
}

// bit length of every segment: one block per group, the stream's code lengths
// in shared memory, a thread per segment
__global__ void __launch_bounds__(256) k_dfl_seglen(DflArgs a) {
    const DflFrame& F = a.fr[blockIdx.y];
    DflScratch& S = *F.S;
    const uint32_t g = blockIdx.x;
    if (S.err || g >= S.ngrp) return;
    const int c = group_stream(S.comp, (int)S.nstr, g);
    const DflComp& C = S.comp[c];
    __shared__ uint8_t len[DFL_NLIT];
    for (int i = threadIdx.x; i < DFL_NLIT; i += blockDim.x) len[i] = S.len[c * DFL_NLIT + i];
    __syncthreads();
    const uint32_t k = (g - C.grp0) * DFL_GRP + threadIdx.x;         // segment inside the stream
    if (C.seg0 + k >= S.comp[c + 1].seg0) return;
    const unsigned long long b0 = (unsigned long long)k * DFL_SEG;
    const unsigned long long b1 = min(C.bytes, b0 + DFL_SEG);
    const uint8_t* p = F.in + C.in_off;
    uint32_t bits = 0;
    for (unsigned long long i = b0; i < b1; i++) bits += len[p[i]];
    S.segbits[C.seg0 + k] = bits;
}

// zero the words of the stream region (the streams are OR-ed in)
__global__ void k_dfl_zero(DflArgs a) {
    const DflFrame& F = a.fr[blockIdx.y];
    DflScratch& S = *F.S;
    if (S.err) return;
    uint32_t* w = reinterpret_cast<uint32_t*>(F.out);
    const unsigned long long w0 = S.streams >> 2, w1 = (S.total - S.tail + 3) >> 2;
    for (unsigned long long i = w0 + blockIdx.x * blockDim.x + threadIdx.x; i < w1; i += gridDim.x * blockDim.x)
        w[i] = 0;
}

// OR n <= 32 bits into the word array at absolute bit position ab
__device__ __forceinline__ void or_bits(uint32_t* w, unsigned long long ab, uint32_t v, int n) {
    if (n == 0) return;
    const unsigned long long x = (unsigned long long)v << (ab & 31);
    atomicOr(&w[ab >> 5], (uint32_t)x);
    if ((int)(ab & 31) + n > 32) atomicOr(&w[(ab >> 5) + 1], (uint32_t)(x >> 32));
}

// the data of every segment: one block per group, the stream's codes in
// shared memory, a thread per segment; the first group's thread 0 adds the
// header, the thread of the last segment the end-of-block code
__global__ void __launch_bounds__(256) k_dfl_write(DflArgs a) {
    const DflFrame& F = a.fr[blockIdx.y];
    DflScratch& S = *F.S;
    const uint32_t g = blockIdx.x;
    if (S.err || g >= S.ngrp) return;
    const int c = group_stream(S.comp, (int)S.nstr, g);
    const DflComp& C = S.comp[c];
    __shared__ uint8_t len[DFL_NLIT];
    __shared__ uint16_t code[DFL_NLIT];
    for (int i = threadIdx.x; i < DFL_NLIT; i += blockDim.x) {
        len[i] = S.len[c * DFL_NLIT + i];
        code[i] = S.code[c * DFL_NLIT + i];
    }
    __syncthreads();
    uint32_t* w = reinterpret_cast<uint32_t*>(F.out);
    const unsigned long long base = 8ULL * C.out_off;
    if (g == C.grp0 && threadIdx.x == 0) {
        const uint8_t* hb = S.hdr + (size_t)c * DFL_HDR_BYTES;
        for (uint32_t b = 0; b < C.hdr_bits; b += 8) or_bits(w, base + b, hb[b >> 3], (int)min(8u, C.hdr_bits - b));
    }
    const uint32_t nseg = S.comp[c + 1].seg0 - C.seg0;
    const uint32_t k = (g - C.grp0) * DFL_GRP + threadIdx.x;
    if (k >= nseg) return;
    const uint32_t s = C.seg0 + k;
    // segment bit offset inside the stream: the header, then the earlier segments
    const unsigned long long ab = base + C.hdr_bits + (S.segoff[s] - S.segoff[C.seg0]);
    const unsigned long long b0 = (unsigned long long)k * DFL_SEG;
    const unsigned long long b1 = min(C.bytes, b0 + DFL_SEG);
    const uint8_t* p = F.in + C.in_off;
    // accumulate into whole words, OR-ed at the word grid
    unsigned long long acc = 0;
    int nacc = (int)(ab & 31);
    unsigned long long wi = ab >> 5;
    auto emit = [&](uint32_t v, int n) {
        acc |= (unsigned long long)v << nacc;
        nacc += n;
        if (nacc >= 32) {
            atomicOr(&w[wi++], (uint32_t)acc);
            acc >>= 32;
            nacc -= 32;
        }
    };
    for (unsigned long long i = b0; i < b1; i++) emit(code[p[i]], len[p[i]]);
    if (k + 1 == nseg) emit(code[256], len[256]);
    if (nacc > 0) atomicOr(&w[wi], (uint32_t)acc);
}

// container tables and the motion vectors (after the streams are written)
__global__ void k_dfl_tables(DflArgs a) {
    const DflFrame& F = a.fr[blockIdx.y];
    DflScratch& S = *F.S;
    if (S.err) return;
    const int t = blockIdx.x * blockDim.x + threadIdx.x, nt = gridDim.x * blockDim.x;
    uint8_t* o = F.out;
    // version 2: a stream per component; 3: one stream (CVC-NTS)
    for (int i = t; i < (int)a.hdr_bytes; i += nt) o[i] = i == 4 ? (a.nts ? 3 : 2) : F.in[i];
    const int nstr = (int)S.nstr;
    for (int c = t; c < nstr; c += nt) wr32(o + a.hdr_bytes + 4 * c, (uint32_t)S.comp[c].out_bytes);
    uint8_t* st = o + a.hdr_bytes + 4 * nstr;
    for (uint32_t s = t; s < S.nseg; s += nt) {
        st[2 * s] = (uint8_t)S.segbits[s];
        st[2 * s + 1] = (uint8_t)(S.segbits[s] >> 8);
    }
    for (uint32_t s = 2 * S.nseg + t; s < ((2 * S.nseg + 3) & ~3u); s += nt) st[s] = 0;
    const unsigned long long tail_in = a.hdr_bytes + S.tok_bytes, tail_out = S.total - S.tail;
    for (unsigned long long i = t; i < S.tail; i += nt) o[tail_out + i] = F.in[tail_in + i];
}

// -------------------------------------------------------------- inflate
// the container's tables: token offsets, segments, groups, stream offsets
// (one block per frame).  Version 2: a stream per component; 3: one stream.
__global__ void __launch_bounds__(256) k_ifl_plan(DflArgs a) {
    const DflFrame& F = a.fr[blockIdx.y];
    DflScratch& S = *F.S;
    __shared__ unsigned long long sh[8];
    __shared__ int s_bad, s_one;
    const uint8_t* in = F.in;
    if (threadIdx.x == 0) {
        S.err = 0;
        S.total = 0;
        s_bad = F.in_len < (long long)a.hdr_bytes || rd32(in) != 0x31435643u || (in[4] != 2 && in[4] != 3) ||
                in[5] > 5 || rd32(in + 28) != (uint32_t)a.ncomp;
        s_one = !s_bad && in[4] == 3;
        if (!s_bad && F.in_len < a.hdr_bytes + 4LL * (s_one ? 1 : a.ncomp)) s_bad = 1;
        if (s_bad) S.err = DFL_CORRUPT;
    }
    __syncthreads();
    if (s_bad) return;
    const int one = s_one, nstr = one ? 1 : a.ncomp;
    const unsigned long long tabs = a.hdr_bytes + 4ULL * nstr;
    unsigned long long tok = 0, seg = 0, grp = 0, sb = 0, tt, ts, tg, tb;
    for (int b = 0; b < a.ncomp; b += blockDim.x) {
        const int c = b + threadIdx.x;
        const uint32_t n = c < a.ncomp ? rd32(in + 32 + 4 * c) : 0;
        const uint32_t nb = c < a.ncomp && !one ? rd32(in + a.hdr_bytes + 4 * c) : 0;
        const unsigned long long segs = one ? 0 : (2ULL * n + DFL_SEG - 1) / DFL_SEG;
        const unsigned long long grps = (segs + DFL_GRP - 1) / DFL_GRP;
        const unsigned long long pt = block_scan(n, sh, &tt), ps = block_scan(segs, sh, &ts),
                                 pg = block_scan(grps, sh, &tg), pb = block_scan(nb, sh, &tb);
        if (c < a.ncomp && !one) {
            S.comp[c].bytes = 2ULL * n;
            S.comp[c].in_off = a.hdr_bytes + 2 * (tok + pt);   // in the inflated frame
            S.comp[c].seg0 = (uint32_t)(seg + ps);
            S.comp[c].grp0 = (uint32_t)(grp + pg);
            S.comp[c].out_off = sb + pb;                     // relative to the streams, fixed below
            S.comp[c].out_bytes = nb;
            if ((nb == 0) != (n == 0)) atomicOr(&S.err, DFL_CORRUPT);
        }
        tok += tt;
        seg += ts;
        grp += tg;
        sb += tb;
    }
    if (one) {
        seg = (2 * tok + DFL_SEG - 1) / DFL_SEG;
        grp = (seg + DFL_GRP - 1) / DFL_GRP;
        sb = rd32(in + a.hdr_bytes);
        if (threadIdx.x == 0) {
            S.comp[0].bytes = 2 * tok;
            S.comp[0].in_off = a.hdr_bytes;
            S.comp[0].seg0 = 0;
            S.comp[0].grp0 = 0;
            S.comp[0].out_off = 0;
            S.comp[0].out_bytes = sb;
            if ((sb == 0) != (tok == 0)) atomicOr(&S.err, DFL_CORRUPT);
        }
    }
    __syncthreads();
    const unsigned long long streams = tabs + ((2ULL * seg + 3) & ~3ULL);
    if (seg <= (unsigned long long)a.max_seg)
        for (int c = threadIdx.x; c < nstr; c += blockDim.x) S.comp[c].out_off += streams;
    if (threadIdx.x == 0) {
        S.comp[nstr].seg0 = (uint32_t)seg;
        S.comp[nstr].grp0 = (uint32_t)grp;
        const long long mvb = in[6] == 2 ? a.mv_bytes : 0;
        if (seg > (unsigned long long)a.max_seg || grp > (unsigned long long)a.max_grp ||
            (in[6] == 2 && a.mv_bytes == 0) || streams + sb + mvb > (unsigned long long)F.in_len)
            atomicOr(&S.err, DFL_CORRUPT);
        S.nseg = (uint32_t)seg;
        S.nstr = (uint32_t)nstr;
        S.ngrp = (uint32_t)grp;
        S.tok_bytes = 2 * tok;
        S.tail = mvb;
        S.streams = streams + sb;                  // where the motion vectors start
        S.total = a.hdr_bytes + 2 * tok + mvb;
        if (S.total > (unsigned long long)F.out_cap) atomicOr(&S.err, DFL_CAPACITY);
    }
}

// segment bit lengths from the container
__global__ void k_ifl_seglen(DflArgs a) {
    const DflFrame& F = a.fr[blockIdx.y];
    DflScratch& S = *F.S;
    const uint32_t s = blockIdx.x * blockDim.x + threadIdx.x;
    if (S.err || s >= (uint32_t)a.max_seg) return;
    if (s >= S.nseg) {
        S.segbits[s] = 0;
        return;
    }
    const uint8_t* st = F.in + a.hdr_bytes + 4 * S.nstr;
    S.segbits[s] = (uint32_t)st[2 * s] | ((uint32_t)st[2 * s + 1] << 8);
}

// block header of each stream -> decoding tables (one block per stream):
// the header is read by one thread; the canonical code then
// fills a 2^DFL_LUT-entry table indexed by the next DFL_LUT bits of the
// stream (symbol | length << 9; 0 for longer codes, which take the
// bit-serial canonical decoder)
__global__ void __launch_bounds__(128) k_ifl_tables(DflArgs a) {
    const DflFrame& F = a.fr[blockIdx.y];
    DflScratch& S = *F.S;
    const int c = blockIdx.x, tid = threadIdx.x;
    if (S.err || c >= (int)S.nstr) return;
    DflComp& C = S.comp[c];
    if (C.bytes == 0) return;
    __shared__ uint8_t lens[286 + 30];
    __shared__ int s_ok, s_hlit;
    __shared__ uint16_t nextc[16];
    __shared__ uint8_t head[DFL_HDR_BYTES];     // a valid block header fits
    const unsigned long long nh = min((unsigned long long)DFL_HDR_BYTES, C.out_bytes);
    for (unsigned long long i = tid; i < nh; i += blockDim.x) head[i] = F.in[C.out_off + i];
    __syncthreads();
    if (tid == 0) {
        // bits of the header, LSB first, from shared memory through a 64-bit buffer
        unsigned long long buf = 0, bp = 0, pos = 0;
        const unsigned long long hbits = 8ULL * nh;
        int nb = 0;
        bool bad = false;
        auto get = [&](int n) -> uint32_t {
            while (nb < n) {
                buf |= (unsigned long long)(bp < nh ? head[bp] : 0) << nb;
                bp++;
                nb += 8;
            }
            const uint32_t v = (uint32_t)(buf & ((1ull << n) - 1));
            buf >>= n;
            nb -= n;
            pos += n;
            if (pos > hbits) bad = true;
            return v;
        };
        const uint32_t bfinal = get(1), btype = get(2);
        const int hlit = (int)get(5) + 257, hdist = (int)get(5) + 1, hclen = (int)get(4) + 4;
        bool ok = bfinal == 1 && btype == 2 && hlit <= 286 && hdist <= 30;
        uint8_t cl[19] = {0};
        for (int i = 0; i < hclen; i++) cl[CL_ORDER[i]] = (uint8_t)get(3);
        // code-length code: 7-bit lookup table, symbol | length << 5 (0: no code)
        uint16_t lut[128];
        for (int i = 0; i < 128; i++) lut[i] = 0;
        {
            int cnt[8] = {0}, left = 1;
            for (int i = 0; i < 19; i++) cnt[cl[i]]++;
            cnt[0] = 0;
            for (int b = 1; b < 8; b++) {
                left = (left << 1) - cnt[b];
                if (left < 0) ok = false;
            }
            int nc[8], cc = 0;
            for (int b = 1; b < 8; b++) {
                cc = (cc + cnt[b - 1]) << 1;
                nc[b] = cc;
            }
            for (int i = 0; ok && i < 19; i++) {
                const int l = cl[i];
                if (!l) continue;
                const uint32_t rc = bit_reverse((uint32_t)nc[l]++, l);
                for (uint32_t k = 0; k < (1u << (7 - l)); k++) lut[rc | (k << l)] = (uint16_t)(i | (l << 5));
            }
        }
        const int n = hlit + hdist;
        for (int i = 0; ok && i < n;) {
            while (nb < 7) {
                buf |= (unsigned long long)(bp < nh ? head[bp] : 0) << nb;
                bp++;
                nb += 8;
            }
            const uint16_t e = lut[buf & 127];
            if (!e) { ok = false; break; }
            const int sym = e & 31, l = e >> 5;
            buf >>= l;
            nb -= l;
            pos += l;
            if (pos > hbits) { ok = false; break; }
            if (sym < 16) {
                lens[i++] = (uint8_t)sym;
                continue;
            }
            int rep, val = 0;
            if (sym == 16) {
                if (i == 0) { ok = false; break; }
                val = lens[i - 1];
                rep = 3 + (int)get(2);
            } else if (sym == 17) {
                rep = 3 + (int)get(3);
            } else {
                rep = 11 + (int)get(7);
            }
            if (i + rep > n) { ok = false; break; }
            while (rep-- > 0) lens[i++] = (uint8_t)val;
        }
        ok = ok && !bad;
        uint8_t ll[286];
        for (int i = 0; ok && i < hlit; i++) ll[i] = lens[i];
        ok = ok && lens[256] != 0 && build_decoder(ll, hlit, S.dcount + c * 16, S.dsym + c * DFL_NSYM);
        if (ok) {
            uint16_t cnt[16] = {0};
            for (int i = 0; i < hlit; i++) cnt[lens[i]]++;
            cnt[0] = 0;
            uint16_t cc = 0;
            for (int b = 1; b < 16; b++) {
                cc = (uint16_t)((cc + cnt[b - 1]) << 1);
                nextc[b] = cc;
            }
            C.hdr_bits = (uint32_t)pos;
        } else {
            atomicOr(&S.err, DFL_CORRUPT);
        }
        s_ok = ok;
        s_hlit = hlit;
    }
    __syncthreads();
    if (!s_ok) return;
    uint16_t* tab = S.dtab + (size_t)c * (1 << DFL_LUT);
    for (int i = tid; i < (1 << DFL_LUT); i += blockDim.x) tab[i] = 0;
    __syncthreads();
    for (int i = tid; i < s_hlit; i += blockDim.x) {
        const int l = lens[i];
        if (l == 0 || l > DFL_LUT) continue;
        int r = 0;
        for (int j = 0; j < i; j++) r += lens[j] == l;
        const uint32_t rc = bit_reverse(nextc[l] + r, l);
        for (uint32_t k = 0; k < (1u << (DFL_LUT - l)); k++) tab[rc | (k << l)] = (uint16_t)(i | (l << 9));
    }
}

// the literals of every segment: one block per group, the stream's decoding
// tables in shared memory, one thread per segment (lookup table, longer codes
// bit by bit); each segment must take exactly its recorded bits, and the
// stream's last one must be followed by the end-of-block code
__global__ void __launch_bounds__(256) k_ifl_decode(DflArgs a) {
    const DflFrame& F = a.fr[blockIdx.y];
    DflScratch& S = *F.S;
    const uint32_t g = blockIdx.x;
    if (S.err || g >= S.ngrp) return;
    const int c = group_stream(S.comp, (int)S.nstr, g);
    const DflComp& C = S.comp[c];
    __shared__ uint16_t tab[1 << DFL_LUT];
    __shared__ uint16_t count[16], sym[DFL_NSYM];
    for (int i = threadIdx.x; i < (1 << DFL_LUT); i += blockDim.x) tab[i] = S.dtab[(size_t)c * (1 << DFL_LUT) + i];
    for (int i = threadIdx.x; i < DFL_NSYM; i += blockDim.x) sym[i] = S.dsym[c * DFL_NSYM + i];
    if (threadIdx.x < 16) count[threadIdx.x] = S.dcount[c * 16 + threadIdx.x];
    __syncthreads();
    const uint8_t* p = F.in + C.out_off;
    const unsigned long long nbytes = C.out_bytes, end = 8ULL * nbytes;
    uint8_t* o = F.out + C.in_off;
    const uint32_t nseg = S.comp[c + 1].seg0 - C.seg0;
    bool ok = true;
    const uint32_t k = (g - C.grp0) * DFL_GRP + threadIdx.x;
    if (k < nseg) {
        const uint32_t s = C.seg0 + k;
        const unsigned long long start = C.hdr_bits + (S.segoff[s] - S.segoff[C.seg0]);
        const unsigned long long stop = start + S.segbits[s];
        // bit buffer: buf holds nb bits, the next of them at bit 0; bytes past the stream read as 0
        unsigned long long buf = 0, bp = start >> 3, pos = start;
        int nb = 0;
        // four independent byte loads per refill, so that their latencies overlap
        auto refill = [&]() {
            uint32_t x = 0;
#pragma unroll
            for (int k = 0; k < 4; k++) x |= (uint32_t)(bp + k < nbytes ? p[bp + k] : 0) << (8 * k);
            buf |= (unsigned long long)x << nb;
            bp += 4;
            nb += 32;
        };
        refill();
        buf >>= (start & 7);
        nb -= (int)(start & 7);
        auto next = [&]() -> int {
            if (nb < 16) refill();
            const uint16_t e = tab[buf & ((1u << DFL_LUT) - 1)];
            if (e) {
                const int l = e >> 9;
                buf >>= l;
                nb -= l;
                pos += l;
                return e & 511;
            }
            int code = 0, first = 0, index = 0;
            for (int l = 1; l <= 15; l++) {
                code |= (int)(buf & 1);
                buf >>= 1;
                nb--;
                pos++;
                const int n = count[l];
                if (code - first < n) return sym[index + code - first];
                index += n;
                first = (first + n) << 1;
                code <<= 1;
            }
            return -1;
        };
        const unsigned long long b0 = (unsigned long long)k * DFL_SEG;
        const unsigned long long b1 = min(C.bytes, b0 + DFL_SEG);
        for (unsigned long long i = b0; i < b1; i++) {
            const int v = next();
            if (v < 0 || v > 255) { ok = false; break; }
            o[i] = (uint8_t)v;
        }
        ok = ok && pos == stop && pos <= end;
        if (ok && k + 1 == nseg) ok = next() == 256 && pos <= end;
    }
    if (!ok) atomicOr(&S.err, DFL_CORRUPT);
}

__global__ void k_ifl_finish(DflArgs a) {
    const DflFrame& F = a.fr[blockIdx.y];
    DflScratch& S = *F.S;
    if (S.err) return;
    const int t = blockIdx.x * blockDim.x + threadIdx.x, nt = gridDim.x * blockDim.x;
    uint8_t* o = F.out;
    for (int i = t; i < (int)a.hdr_bytes; i += nt) o[i] = i == 4 ? 1 : F.in[i];
    const unsigned long long tail_out = a.hdr_bytes + S.tok_bytes;
    for (unsigned long long i = t; i < S.tail; i += nt) o[tail_out + i] = F.in[S.streams + i];
}

}  // namespace cvc
