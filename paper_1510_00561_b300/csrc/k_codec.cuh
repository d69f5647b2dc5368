// k_codec.cuh -- parameter blocks and kernels of the codec stages.
#pragma once
#include "cvc_internal.cuh"

namespace cvc {

struct ColourGeom {
    int H, W;      // frame
    int Hp, Wp;    // padded luma plane
    int Hc, Wc;    // 4:2:0 chroma
    int Hcp, Wcp;  // padded chroma plane
};

// coefficient frame: planes Y, Co, Cg back to back, lowpass first in each
struct FrameGeom {
    long long poff[3];   // plane offsets
    long long low_n[3];  // lowpass elements per plane
    int low_w[3];        // lowpass row length per plane
    long long total;
};

struct QuantParams {
    float qph, qpl;
    float threshold;
    float low_scale;    // 2^-L (exact)
    float qpl_denorm;   // qpl * 2^L (exact)
};

// rows of every component in stream order
struct RowTable {
    const long long* off;   // element offset of the row in the frame
    const int* w;           // row length
    const uint8_t* low;     // row belongs to a lowpass component
    int nrows;
};

struct StreamHeader {
    int type, levels;
    uint32_t frame_index;
    int height, width;
    int dirs[6];
    int qph, qpl;
};

struct DecInfo {
    int type;
    uint32_t frame_index;
    uint32_t total;   // tokens in the stream (0 if the header is bad)
    uint32_t pad;
};

__global__ void k_colour_fwd(const uint8_t* rgb, long long pitch, ColourGeom g, float* Y, float* Co, float* Cg);
__global__ void k_colour_inv(const float* Y, const float* Co, const float* Cg, ColourGeom g, uint8_t* rgb,
                             long long pitch);
__global__ void k_quant(const float* coef, const int16_t* prev, FrameGeom f, QuantParams qp, int is_key,
                        int16_t* q_out, int16_t* r_out, uint32_t* err);
__global__ void k_unquant(const int16_t* res, const int16_t* prev, FrameGeom f, QuantParams qp, const DecInfo* info,
                          int16_t* q_out, float* coef);
__global__ void k_unquant_keylow(const int16_t* res, FrameGeom f, QuantParams qp, const DecInfo* info,
                                 int16_t* q_out, float* coef);
__global__ void k_rle_count(const int16_t* res, const RowTable rt, int is_key, uint32_t* cnt);
__global__ void k_rle_write(const int16_t* res, const RowTable rt, int is_key, const uint32_t* tokoff,
                            uint8_t* tok_base, uint32_t cap_tok, uint32_t* err);
__global__ void k_stream_header(StreamHeader h, const uint32_t* tokoff, const int* comp_row0, int ncomp,
                                uint8_t* out, uint32_t* info);
__global__ void k_dec_parse(const uint8_t* in, long long in_len, StreamHeader expect, int ncomp, long long expect_next,
                            uint32_t max_tok, uint32_t* comp_tok, DecInfo* info, uint32_t* err);
__global__ void k_dec_contrib(const uint8_t* tok, const uint32_t* comp_tok, int ncomp, const uint8_t* comp_low,
                              const DecInfo* info, uint32_t* contrib, uint32_t max_tok, uint32_t* err);
__global__ void k_dec_check(const uint32_t* comp_tok, const uint32_t* pos, const long long* comp_elem, int ncomp,
                            const DecInfo* info, uint32_t* err);
__global__ void k_dec_scatter(const uint8_t* tok, const uint32_t* comp_tok, int ncomp, const uint8_t* comp_low,
                              const DecInfo* info, const uint32_t* pos, long long ncoef, int16_t* res);

// exclusive scan of n values into out[0..n] (out[n] = total); tmp holds
// ceil(n / 2048) + 1 values.
cudaError_t exclusive_scan(const uint32_t* in, uint32_t n, uint32_t* out, uint32_t* tmp, cudaStream_t st);

}  // namespace cvc
