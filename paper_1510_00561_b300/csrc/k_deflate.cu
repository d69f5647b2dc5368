// k_deflate.cu -- the DEFLATE stage of CVC (§3.9), scalable mode: every
// component's token bytes become one raw DEFLATE stream (RFC 1951) of its
// own, so that a receiver can be sent any subset of components.
//
// Each stream is one final block with dynamic Huffman codes over literal
// bytes only (the Huffman-only strategy: no LZ77 matches), which makes both
// directions data-parallel:
//   deflate  a byte histogram per component, one length-limited Huffman code
//            per component (one thread each), the block header, and the
//            data written by one thread per 256-byte segment at a bit offset
//            from a scan of the segments' bit lengths;
//   inflate  one thread per component decodes its block header into
//            canonical decoding tables, one thread per segment decodes its
//            256 literals starting at the bit offset the container records.
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

// Huffman code lengths of n symbols (weights w, 0 = unused) limited to
// maxlen bits.  A binary heap of (weight, node) builds the tree; if it is too
// deep, the weights are halved (non-zero ones stay >= 1) and it is built
// again.  A lone used symbol gets one bit.
__device__ void huffman_lengths(const uint32_t* w_in, int n, int maxlen, uint8_t* len, uint32_t* w, uint16_t* parent,
                                uint16_t* heap) {
    int used = 0;
    for (int i = 0; i < n; i++) {
        w[i] = w_in[i];
        len[i] = 0;
        used += w_in[i] != 0;
    }
    if (used < 2) {                    // a lone symbol gets one bit (the caller completes the code)
        for (int i = 0; i < n; i++) len[i] = w_in[i] ? 1 : 0;
        return;
    }
    for (;;) {
        int hn = 0, m = n;
        auto less = [&](int a, int b) { return w[a] < w[b] || (w[a] == w[b] && a < b); };
        auto push = [&](int x) {
            int i = hn++;
            heap[i] = (uint16_t)x;
            while (i > 0) {
                int p = (i - 1) >> 1;
                if (!less(heap[i], heap[p])) break;
                uint16_t t = heap[i]; heap[i] = heap[p]; heap[p] = t;
                i = p;
            }
        };
        auto pop = [&]() {
            int top = heap[0];
            heap[0] = heap[--hn];
            int i = 0;
            for (;;) {
                int l = 2 * i + 1, r = l + 1, s = i;
                if (l < hn && less(heap[l], heap[s])) s = l;
                if (r < hn && less(heap[r], heap[s])) s = r;
                if (s == i) break;
                uint16_t t = heap[i]; heap[i] = heap[s]; heap[s] = t;
                i = s;
            }
            return top;
        };
        for (int i = 0; i < n; i++)
            if (w[i]) push(i);
        while (hn > 1) {
            int a = pop(), b = pop();
            w[m] = w[a] + w[b];
            parent[a] = parent[b] = (uint16_t)m;
            push(m);
            m++;
        }
        const int root = m - 1;
        int deepest = 0;
        for (int i = 0; i < n; i++) {
            int d = 0;
            if (w_in[i]) {
                for (int x = i; x != root; x = parent[x]) d++;
            }
            len[i] = (uint8_t)d;
            deepest = max(deepest, d);
        }
        if (deepest <= maxlen) return;
        for (int i = 0; i < n; i++) w[i] = w[i] ? (w[i] + 1) >> 1 : 0;
    }
}

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
    uint32_t pos, cap;
    bool over;
    __device__ void put(uint32_t v, int n) {
        for (int i = 0; i < n; i++) {
            if (pos >= cap) { over = true; return; }
            if ((v >> i) & 1u) p[pos >> 3] |= (uint8_t)(1u << (pos & 7));
            pos++;
        }
    }
};

// sequential bit reader over [0, nbits)
struct BitIn {
    const uint8_t* p;
    unsigned long long pos, end;
    bool bad;
    __device__ uint32_t get(int n) {
        uint32_t v = 0;
        for (int i = 0; i < n; i++) {
            if (pos >= end) { bad = true; return 0; }
            v |= (uint32_t)((p[pos >> 3] >> (pos & 7)) & 1u) << i;
            pos++;
        }
        return v;
    }
};

// canonical decoding: the code of a symbol is read MSB first, one bit at a time.
// This and build_decoder stay out of line: inlined into k_ifl_tables with its
// local tables, our sm_103a build decoded wrong code-length symbols, while the
// same source run on the host and the out-of-line form decode correctly.
__device__ __noinline__ int decode_sym(BitIn& in, const uint16_t* count, const uint16_t* sym) {
    int code = 0, first = 0, index = 0;
    for (int len = 1; len <= 15; len++) {
        code |= (int)in.get(1);
        const int c = count[len];
        if (code - first < c) return sym[index + code - first];
        index += c;
        first = (first + c) << 1;
        code <<= 1;
    }
    in.bad = true;
    return -1;
}

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

}  // namespace

// -------------------------------------------------------------- deflate
// one thread: component byte offsets of the input tokens and the segments
__global__ void k_dfl_plan(DflArgs a) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    DflScratch& S = *a.S;
    S.err = 0;
    S.total = 0;
    const uint8_t* in = a.in;
    if (a.in_len < (long long)a.hdr_bytes || rd32(in) != 0x31435643u || in[4] != 1 || in[5] != 0 ||
        rd32(in + 28) != (uint32_t)a.ncomp) {
        S.err = DFL_CORRUPT;
        return;
    }
    unsigned long long tok = 0;
    uint32_t seg = 0;
    for (int c = 0; c < a.ncomp; c++) {
        const uint32_t n = rd32(in + 32 + 4 * c);
        S.comp[c].in_off = a.hdr_bytes + 2 * tok;
        S.comp[c].bytes = 2 * n;
        S.comp[c].seg0 = seg;
        tok += n;
        seg += (2 * n + DFL_SEG - 1) / DFL_SEG;
    }
    S.comp[a.ncomp].seg0 = seg;
    const int type = in[6];
    const long long mvb = type == 2 ? a.mv_bytes : 0;
    if ((type == 2 && a.mv_bytes == 0) || seg > (uint32_t)a.max_seg || a.hdr_bytes + 2 * tok + mvb > (unsigned long long)a.in_len) {
        S.err = DFL_CORRUPT;
        return;
    }
    S.nseg = seg;
    S.tok_bytes = 2 * tok;
    S.tail = mvb;
}

// byte histogram of each component: one block per component
__global__ void __launch_bounds__(256) k_dfl_hist(DflArgs a) {
    DflScratch& S = *a.S;
    if (S.err) return;
    const int c = blockIdx.x;
    __shared__ uint32_t h[256];
    for (int i = threadIdx.x; i < 256; i += blockDim.x) h[i] = 0;
    __syncthreads();
    const uint8_t* p = a.in + S.comp[c].in_off;
    const unsigned long long n = S.comp[c].bytes;
    for (unsigned long long i = threadIdx.x; i < n; i += blockDim.x) atomicAdd(&h[p[i]], 1u);
    __syncthreads();
    for (int i = threadIdx.x; i < 256; i += blockDim.x) S.hist[c * DFL_NLIT + i] = h[i];
    if (threadIdx.x == 0) S.hist[c * DFL_NLIT + 256] = 1;   // end of block
}

// code of each component (one thread per component): literal/length code
// lengths and codes, the run-length coded header, its bit length
__global__ void k_dfl_code(DflArgs a) {
    DflScratch& S = *a.S;
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (S.err || c >= a.ncomp) return;
    DflComp& C = S.comp[c];
    if (C.bytes == 0) {
        C.hdr_bits = 0;
        C.data_bits = 0;
        return;
    }
    uint32_t w[2 * DFL_NLIT];
    uint16_t parent[2 * DFL_NLIT], heap[DFL_NLIT];
    uint8_t* len = S.len + c * DFL_NLIT;
    huffman_lengths(S.hist + c * DFL_NLIT, DFL_NLIT, 15, len, w, parent, heap);
    canonical_codes(len, DFL_NLIT, S.code + c * DFL_NLIT);
    // code lengths of the 257 literal/length codes and of two (unused) distance
    // codes of one bit, run-length coded with the code-length alphabet
    uint8_t seq[DFL_NLIT + 2];
    for (int i = 0; i < DFL_NLIT; i++) seq[i] = len[i];
    seq[DFL_NLIT] = seq[DFL_NLIT + 1] = 1;
    const int N = DFL_NLIT + 2;
    uint8_t rs[DFL_NLIT + 2], rx[DFL_NLIT + 2];   // code-length symbols, their extra values
    int nr = 0;
    for (int i = 0; i < N;) {
        const int v = seq[i];
        int run = 1;
        while (i + run < N && seq[i + run] == v) run++;
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
    {
        uint32_t w2[38];
        uint16_t p2[38], h2[19];
        huffman_lengths(cf, 19, 7, cl, w2, p2, h2);
    }
    // a single used code-length symbol still needs a complete prefix code: give it a one-bit partner
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
    // the header bits
    uint8_t* hb = S.hdr + (size_t)c * DFL_HDR_BYTES;
    for (int i = 0; i < DFL_HDR_BYTES; i++) hb[i] = 0;
    BitOut o{hb, 0, DFL_HDR_BYTES * 8, false};
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
    if (o.over) S.err = DFL_INTERNAL;
    C.hdr_bits = o.pos;
    unsigned long long bits = 0;
    for (int i = 0; i < DFL_NLIT; i++) bits += (unsigned long long)S.hist[c * DFL_NLIT + i] * len[i];
    C.data_bits = bits;            // the literals and the end-of-block code
}

// one thread: stream offsets, container layout, the size check
__global__ void k_dfl_layout(DflArgs a) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    DflScratch& S = *a.S;
    if (S.err) return;
    const unsigned long long tables = a.hdr_bytes + 4ULL * a.ncomp + ((2ULL * S.nseg + 3) & ~3ULL);
    unsigned long long off = tables;
    for (int c = 0; c < a.ncomp; c++) {
        DflComp& C = S.comp[c];
        C.out_off = off;
        C.out_bytes = C.bytes ? (C.hdr_bits + C.data_bits + 7) >> 3 : 0;
        off += C.out_bytes;
    }
    S.streams = tables;
    S.total = off + S.tail;
    if (S.total > (unsigned long long)a.out_cap) S.err = DFL_CAPACITY;
}

// bit length of every segment (one thread per segment)
__global__ void k_dfl_seglen(DflArgs a) {
    DflScratch& S = *a.S;
    const uint32_t s = blockIdx.x * blockDim.x + threadIdx.x;
    if (S.err || s >= (uint32_t)a.max_seg) return;
    if (s >= S.nseg) {
        S.segbits[s] = 0;
        return;
    }
    int lo = 0, hi = a.ncomp;             // the component with seg0 <= s < seg0 of the next
    while (hi - lo > 1) {
        const int mid = (lo + hi) >> 1;
        if (S.comp[mid].seg0 <= s) lo = mid;
        else hi = mid;
    }
    while (lo + 1 < a.ncomp && S.comp[lo + 1].seg0 <= s) lo++;
    const DflComp& C = S.comp[lo];
    const unsigned long long b0 = (unsigned long long)(s - C.seg0) * DFL_SEG;
    const unsigned long long b1 = min(C.bytes, b0 + DFL_SEG);
    const uint8_t* p = a.in + C.in_off;
    const uint8_t* len = S.len + lo * DFL_NLIT;
    uint32_t bits = 0;
    for (unsigned long long i = b0; i < b1; i++) bits += len[p[i]];
    S.segbits[s] = bits;
    S.segcomp[s] = lo;
}

// zero the words of the stream region (the streams are OR-ed in)
__global__ void k_dfl_zero(DflArgs a) {
    DflScratch& S = *a.S;
    if (S.err) return;
    uint32_t* w = reinterpret_cast<uint32_t*>(a.out);
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

// the data of every segment (one thread each), the header of every component
// (the thread of its first segment), the end-of-block code (its last)
__global__ void k_dfl_write(DflArgs a) {
    DflScratch& S = *a.S;
    const uint32_t s = blockIdx.x * blockDim.x + threadIdx.x;
    if (S.err || s >= S.nseg) return;
    const int c = S.segcomp[s];
    const DflComp& C = S.comp[c];
    uint32_t* w = reinterpret_cast<uint32_t*>(a.out);
    const unsigned long long base = 8ULL * C.out_off;
    const uint8_t* len = S.len + c * DFL_NLIT;
    const uint16_t* code = S.code + c * DFL_NLIT;
    if (s == C.seg0) {
        const uint8_t* hb = S.hdr + (size_t)c * DFL_HDR_BYTES;
        for (uint32_t b = 0; b < C.hdr_bits; b += 8) or_bits(w, base + b, hb[b >> 3], (int)min(8u, C.hdr_bits - b));
    }
    // segment bit offset inside the stream: the header, then the earlier segments
    unsigned long long ab = base + C.hdr_bits + (S.segoff[s] - S.segoff[C.seg0]);
    const unsigned long long b0 = (unsigned long long)(s - C.seg0) * DFL_SEG;
    const unsigned long long b1 = min(C.bytes, b0 + DFL_SEG);
    const uint8_t* p = a.in + C.in_off;
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
    if (s + 1 == S.comp[c + 1].seg0 || s + 1 == S.nseg) emit(code[256], len[256]);
    if (nacc > 0) atomicOr(&w[wi], (uint32_t)acc);
}

// container tables and the motion vectors (after the streams are written)
__global__ void k_dfl_tables(DflArgs a) {
    DflScratch& S = *a.S;
    if (S.err) return;
    const int t = blockIdx.x * blockDim.x + threadIdx.x, nt = gridDim.x * blockDim.x;
    uint8_t* o = a.out;
    for (int i = t; i < (int)a.hdr_bytes; i += nt) o[i] = i == 4 ? 2 : a.in[i];   // version 2: deflated
    for (int c = t; c < a.ncomp; c += nt) wr32(o + a.hdr_bytes + 4 * c, (uint32_t)S.comp[c].out_bytes);
    uint8_t* st = o + a.hdr_bytes + 4 * a.ncomp;
    for (uint32_t s = t; s < S.nseg; s += nt) {
        st[2 * s] = (uint8_t)S.segbits[s];
        st[2 * s + 1] = (uint8_t)(S.segbits[s] >> 8);
    }
    for (uint32_t s = 2 * S.nseg + t; s < ((2 * S.nseg + 3) & ~3u); s += nt) st[s] = 0;
    const unsigned long long tail_in = a.hdr_bytes + S.tok_bytes, tail_out = S.total - S.tail;
    for (unsigned long long i = t; i < S.tail; i += nt) o[tail_out + i] = a.in[tail_in + i];
}

// -------------------------------------------------------------- inflate
__global__ void k_ifl_plan(DflArgs a) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    DflScratch& S = *a.S;
    S.err = 0;
    S.total = 0;
    const uint8_t* in = a.in;
    const unsigned long long tabs = a.hdr_bytes + 4ULL * a.ncomp;
    if (a.in_len < (long long)tabs || rd32(in) != 0x31435643u || in[4] != 2 || in[5] != 0 ||
        rd32(in + 28) != (uint32_t)a.ncomp) {
        S.err = DFL_CORRUPT;
        return;
    }
    unsigned long long tok = 0;
    uint32_t seg = 0;
    for (int c = 0; c < a.ncomp; c++) {
        const uint32_t n = rd32(in + 32 + 4 * c);
        S.comp[c].bytes = 2ULL * n;
        S.comp[c].in_off = a.hdr_bytes + 2 * tok;   // in the inflated frame
        S.comp[c].seg0 = seg;
        tok += n;
        seg += (2 * n + DFL_SEG - 1) / DFL_SEG;
    }
    S.comp[a.ncomp].seg0 = seg;
    if (seg > (uint32_t)a.max_seg) {
        S.err = DFL_CORRUPT;
        return;
    }
    const unsigned long long streams = tabs + ((2ULL * seg + 3) & ~3ULL);
    unsigned long long off = streams;
    for (int c = 0; c < a.ncomp; c++) {
        const uint32_t nb = rd32(in + a.hdr_bytes + 4 * c);
        S.comp[c].out_off = off;                  // the stream in the container
        S.comp[c].out_bytes = nb;
        if ((nb == 0) != (S.comp[c].bytes == 0)) S.err = DFL_CORRUPT;
        off += nb;
    }
    const long long mvb = in[6] == 2 ? a.mv_bytes : 0;
    if ((in[6] == 2 && a.mv_bytes == 0) || off + mvb > (unsigned long long)a.in_len) S.err = DFL_CORRUPT;
    S.nseg = seg;
    S.tok_bytes = 2 * tok;
    S.tail = mvb;
    S.streams = off;                              // where the motion vectors start
    S.total = a.hdr_bytes + 2 * tok + mvb;
    if (!S.err && S.total > (unsigned long long)a.out_cap) S.err = DFL_CAPACITY;
}

// segment bit lengths from the container, with their component
__global__ void k_ifl_seglen(DflArgs a) {
    DflScratch& S = *a.S;
    const uint32_t s = blockIdx.x * blockDim.x + threadIdx.x;
    if (S.err || s >= (uint32_t)a.max_seg) return;
    if (s >= S.nseg) {
        S.segbits[s] = 0;
        return;
    }
    const uint8_t* st = a.in + a.hdr_bytes + 4 * a.ncomp;
    S.segbits[s] = (uint32_t)st[2 * s] | ((uint32_t)st[2 * s + 1] << 8);
    int lo = 0, hi = a.ncomp;
    while (hi - lo > 1) {
        const int mid = (lo + hi) >> 1;
        if (S.comp[mid].seg0 <= s) lo = mid;
        else hi = mid;
    }
    while (lo + 1 < a.ncomp && S.comp[lo + 1].seg0 <= s) lo++;
    S.segcomp[s] = lo;
}

// block header of each component -> canonical decoding tables
__global__ void k_ifl_tables(DflArgs a) {
    DflScratch& S = *a.S;
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (S.err || c >= a.ncomp) return;
    DflComp& C = S.comp[c];
    if (C.bytes == 0) return;
    BitIn in{a.in + C.out_off, 0, 8ULL * C.out_bytes, false};
    const uint32_t bfinal = in.get(1), btype = in.get(2);
    const int hlit = (int)in.get(5) + 257, hdist = (int)in.get(5) + 1, hclen = (int)in.get(4) + 4;
    bool ok = bfinal == 1 && btype == 2 && hlit <= 286 && hdist <= 30;
    uint8_t cl[19] = {0};
    for (int i = 0; i < hclen; i++) cl[CL_ORDER[i]] = (uint8_t)in.get(3);
    uint16_t ccount[16], csym[19];
    ok = ok && build_decoder(cl, 19, ccount, csym);
    uint8_t lens[286 + 30];
    const int n = hlit + hdist;
    for (int i = 0; ok && i < n;) {
        const int sym = decode_sym(in, ccount, csym);
        if (in.bad || sym < 0) { ok = false; break; }
        if (sym < 16) {
            lens[i++] = (uint8_t)sym;
            continue;
        }
        int rep, val = 0;
        if (sym == 16) {
            if (i == 0) { ok = false; break; }
            val = lens[i - 1];
            rep = 3 + (int)in.get(2);
        } else if (sym == 17) {
            rep = 3 + (int)in.get(3);
        } else {
            rep = 11 + (int)in.get(7);
        }
        if (i + rep > n) { ok = false; break; }
        while (rep-- > 0) lens[i++] = (uint8_t)val;
    }
    ok = ok && !in.bad && lens[256] != 0 &&
         build_decoder(lens, hlit, S.dcount + c * 16, S.dsym + c * DFL_NSYM);
    if (!ok) {
        atomicOr(&S.err, DFL_CORRUPT);
        return;
    }
    C.hdr_bits = in.pos;
}

// one thread per segment: its literals, and the end-of-block code after the last one
__global__ void k_ifl_decode(DflArgs a) {
    DflScratch& S = *a.S;
    const uint32_t s = blockIdx.x * blockDim.x + threadIdx.x;
    if (S.err || s >= S.nseg) return;
    const int c = S.segcomp[s];
    const DflComp& C = S.comp[c];
    BitIn in{a.in + C.out_off, C.hdr_bits + (S.segoff[s] - S.segoff[C.seg0]), 8ULL * C.out_bytes, false};
    const unsigned long long end_of_seg = in.pos + S.segbits[s];
    const uint16_t* count = S.dcount + c * 16;
    const uint16_t* sym = S.dsym + c * DFL_NSYM;
    const unsigned long long b0 = (unsigned long long)(s - C.seg0) * DFL_SEG;
    const unsigned long long b1 = min(C.bytes, b0 + DFL_SEG);
    uint8_t* o = a.out + C.in_off;
    bool ok = true;
    for (unsigned long long i = b0; i < b1; i++) {
        const int v = decode_sym(in, count, sym);
        if (in.bad || v < 0 || v > 255) { ok = false; break; }
        o[i] = (uint8_t)v;
    }
    ok = ok && in.pos == end_of_seg;
    if (ok && (s + 1 == S.comp[c + 1].seg0 || s + 1 == S.nseg)) ok = decode_sym(in, count, sym) == 256 && !in.bad;
    if (!ok) atomicOr(&S.err, DFL_CORRUPT);
}

__global__ void k_ifl_finish(DflArgs a) {
    DflScratch& S = *a.S;
    if (S.err) return;
    const int t = blockIdx.x * blockDim.x + threadIdx.x, nt = gridDim.x * blockDim.x;
    uint8_t* o = a.out;
    for (int i = t; i < (int)a.hdr_bytes; i += nt) o[i] = i == 4 ? 1 : a.in[i];
    const unsigned long long tail_out = a.hdr_bytes + S.tok_bytes;
    for (unsigned long long i = t; i < S.tail; i += nt) o[tail_out + i] = a.in[S.streams + i];
}

}  // namespace cvc
