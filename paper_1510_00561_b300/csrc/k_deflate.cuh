// k_deflate.cuh -- the DEFLATE stage (§3.9): device structures of the
// Huffman-only DEFLATE (one stream per component, or per frame for CVC-NTS)
// and its inflate.
#pragma once
#include "k_codec.cuh"

namespace cvc {

constexpr int DFL_SEG = 256;         // input bytes per segment (one thread each)
constexpr int DFL_GRP = 256;         // segments per group (one block each)
constexpr int DFL_NLIT = 257;        // literal bytes and the end-of-block code
constexpr int DFL_NSYM = 288;        // decoding table entries per component
constexpr int DFL_HDR_BYTES = 512;   // room for one dynamic block header
constexpr int DFL_LUT = 11;          // bits of the inflate lookup table

enum : uint32_t { DFL_CORRUPT = 1, DFL_CAPACITY = 2, DFL_INTERNAL = 4 };

struct DflComp {
    unsigned long long in_off;     // token bytes in the raw frame
    unsigned long long bytes;      // token bytes of the component
    unsigned long long out_off;    // the component's stream in the container
    unsigned long long out_bytes;  // its length in bytes
    unsigned long long data_bits;  // literals and end-of-block code
    uint32_t seg0;                 // first segment
    uint32_t hdr_bits;             // dynamic block header
    uint32_t grp0;                 // first group of segments
    uint32_t pad;
};

// device scratch of one frame (sized for the stream's largest frame).  A
// "stream" below is a component (scalable mode) or the whole frame (CVC-NTS).
struct DflScratch {
    DflComp* comp;          // streams + 1
    uint32_t* hist;         // ncomp x DFL_NLIT
    uint8_t* len;           // ncomp x DFL_NLIT code lengths
    uint16_t* code;         // ncomp x DFL_NLIT bit-reversed codes
    uint8_t* hdr;           // ncomp x DFL_HDR_BYTES block headers
    uint16_t* dcount;       // ncomp x 16 decoding: codes per length
    uint16_t* dsym;         // ncomp x DFL_NSYM decoding: symbols by code
    uint16_t* dtab;         // ncomp x 2^DFL_LUT decoding: symbol | length << 9 by the next bits
    uint32_t* segbits;      // max_seg + 1 (the frame's slice of one array for all frames)
    uint32_t* segoff;       // max_seg + 1 (exclusive scan of that array, up to a constant per frame)
    uint32_t err, nseg;
    uint32_t nstr, ngrp;    // streams, groups of segments
    unsigned long long tok_bytes, tail, total, streams;
};

// one frame of a call (grid dimension y)
struct DflFrame {
    const uint8_t* in;
    long long in_len;
    uint8_t* out;
    long long out_cap;
    DflScratch* S;          // device: the frame's scratch
};

struct DflArgs {
    const DflFrame* fr;     // device: one per frame of the call
    long long hdr_bytes;    // 32 + 4 ncomp
    long long mv_bytes;     // motion vectors of a type-2 frame
    int ncomp, max_seg, max_grp;
    int nts;                // deflate: one stream per frame (CVC-NTS) instead of one per component
};

__global__ void k_dfl_plan(DflArgs a);
__global__ void k_dfl_hist(DflArgs a);
__global__ void k_dfl_code(DflArgs a);
__global__ void k_dfl_layout(DflArgs a);
__global__ void k_dfl_seglen(DflArgs a);
__global__ void k_dfl_zero(DflArgs a);
__global__ void k_dfl_write(DflArgs a);
__global__ void k_dfl_tables(DflArgs a);
__global__ void k_ifl_plan(DflArgs a);
__global__ void k_ifl_seglen(DflArgs a);
__global__ void k_ifl_tables(DflArgs a);
__global__ void k_ifl_decode(DflArgs a);
__global__ void k_ifl_finish(DflArgs a);

}  // namespace cvc
