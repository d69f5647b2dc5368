// k_codec.cuh -- parameter blocks and kernels of the codec stages, for a
// batch of independent streams (one or many) handled by every launch.
#pragma once
#include "cvc_internal.cuh"

namespace cvc {

struct ColourGeom {
    int H, W;      // frame
    int Hp, Wp;    // padded luma plane
    int Hc, Wc;    // 4:2:0 chroma
    int Hcp, Wcp;  // padded chroma plane
};

struct QuantParams {
    float qph, qpl;
    float threshold;
    float low_scale;    // 2^-L (exact)
    float qpl_denorm;   // qpl * 2^L (exact)
    int st8;            // 8-bit storage (§3.6): codes clamped to a byte
    // 1/qph, 1/qpl where the step is a power of two (exact, so t * (1/qp) is the
    // correctly rounded t / qp, bit for bit); 0 where the quotient needs a division
    float rqph, rqpl;
};

struct StreamHeader {
    int levels;
    int height, width;
    int dirs[6];
    int qph, qpl;
    int flags;          // header byte 5: bit 0 8-bit storage, bits 1-2 DFB prototype (taps / 2 - 2)
};

// per stream, fixed at creation
struct SDesc {
    ColourGeom cg;
    QuantParams qp;
    StreamHeader hdr;
    long long plane_off;   // floats: padded planes Y, Co, Cg of this stream
    long long nplane;
    long long coef_off;    // coefficients of this stream in the frame buffers
    long long ncoef;
    int row0, nrows;       // its component rows in the row table
    int tile0, ntiles;     // its RLE tiles
    int comp0, ncomp;      // its components in the component table
    long long hdr_bytes;   // 32 + 4 * ncomp
    long long max_tok;     // largest valid token count of one frame
    int blk_colour;        // first block of the stream in the forward colour launch
    // planes Y, Co, Cg inside the stream's coefficients: start, lowpass size, and
    // the elements of levels 1..d (absent from a frame that dropped d levels)
    long long pstart[3];
    long long nlow[3];
    long long absent[CVC_MAX_LEVELS + 1][3];
    // motion (§3.2): search range (0: zero-motion P-frames), 16 x 16 luma blocks,
    // the stream's vectors in the vector buffer, its luma planes in the luma buffers,
    // its first block in the motion search launch
    int mv_range, nby, nbx, blk_motion;
    long long mv_off;      // first block's (dy, dx) pair
    long long luma_off;    // bytes
    long long mv_bytes;    // 2 * nby * nbx
    int key_interval;      // frame i is a K-frame iff i % key_interval == 0 (§3.7)
};

// the decoder's output stage of one stream at pyramid scale s (s = 0: full
// resolution).  Scale s reconstructs the level-s lowpass image of every
// plane: the frame and its 4:2:0 chroma shrink to ceil(n / 2^s).
struct ScaleDesc {
    int H, W;              // output frame at this scale
    int Hc, Wc;            // its 4:2:0 chroma
    int rs_y, rs_c;        // row pitch of the luma / chroma planes read
    int src;               // 0: reconstructed planes; 1: the decoded lowpass bands themselves (s = L)
    int blk0;              // first block (output row) of the stream
    long long off[3];      // Y, Co, Cg in that buffer
    float norm;            // 2^-s: the DC gain of s pyramid levels (exact)
    int st8;               // 8-bit storage: Table I colour with chroma offset by 127
};

// per stream, refreshed every call.  The host fills the buffers and switches;
// the step's first kernel (k_step_begin) fills the coder-state fields (ecur ..
// dec_floor) from the stream's device-resident SCtl.
struct SCall {
    const uint8_t* rgb_in;
    long long pitch_in;
    uint8_t* out;
    long long out_cap;
    const uint8_t* in;
    long long in_len;      // < 0: the encoder's output of this call (fused encode + decode)
    uint8_t* rgb_out;
    long long pitch_out;
    int enc_on, enc_key, ecur, dec_on;
    uint32_t enc_index;
    int dcur;
    long long dec_expect;  // frame index a P-frame must carry; -1: a K-frame is required
    int dec_scale;         // pyramid scale of the decoder's output (its buffer was checked for it)
    int dec_floor;         // finest levels 1..dec_floor of the decoder state are missing
    int reset;             // reset the stream's coder state before this step (cvc_reset)
    int no_commit;         // leave the coder state as it was (autotuner runs)
    int async;             // an asynchronous call: its first error is kept in SCtl::first_err
    int pad;
    const size_t* in_len_dev;         // non-NULL: the decoder's input length, read on the device
                                      // (at most in_len, the capacity of the input buffer)
    size_t* out_len_dev;              // non-NULL: where the device writes the encoded length
    int* type_dev;                    // non-NULL: where the device writes the encoded frame type
    cvc_status* enc_status_dev;       // non-NULL: where the device writes the encoder's status
    cvc_status* dec_status_dev;       // non-NULL: where the device writes the decoder's status
    cvc_batch_result* res_dev;        // non-NULL: where the device writes the stream's whole result
};

// per stream, written by the device every call
struct SResult {
    uint32_t enc_err, dec_err;
    uint32_t enc_tokens;     // tokens of the encoded frame
    uint32_t dec_type, dec_index, dec_tokens;
    uint32_t dec_drop;       // finest levels the decoded frame left out
    uint32_t pad;
    cvc_batch_result res;    // the call's outcome (k_step_commit)
};

// per stream, resident on the device: the coder state that decides each
// call's frame type, the state buffers' parity and the decoder's checks.  A
// step reads it first (k_step_begin) and updates it last (k_step_commit) only
// where the call succeeded, so that calls can be queued without host work
// between them.
struct SCtl {
    long long enc_frame;     // the encoder's next frame index
    long long dec_next;      // frame index the decoder's next P-frame must carry; -1: a K-frame is required
    int ecur, dcur;          // which of the two state buffers holds the current codes
    int dec_floor;           // finest levels whose decoder state is missing (dropped in transmission)
    int first_err;           // first non-OK status of an asynchronous call since the last read (cvc_get_error)
};

// per plane (three per stream)
struct PDesc {
    long long coef_off;   // global coefficient offset of the plane
    long long total;
    long long low_n;      // lowpass elements
    int low_w;            // lowpass row length
    int stream;
    int first_block;      // first block of the plane in element-wise launches
    int pad;
};

struct RowTable {
    const long long* off;   // global coefficient index of the row's first element
    const int* w;
    const uint8_t* low;     // row belongs to a lowpass component
    const int* stream;
    const int* comp;        // global component index
    const int4* mc;         // motion compensation: the row's index and the height of its component, ey, ex
    int nrows;
};

// RLE work units: whole rows of one component (all of one width), in stream
// order; at most RLE_TILE codes unless a single row is longer
struct RleTiles {
    const long long* off;     // global coefficient index of the tile's first code
    const int* n;             // codes
    const int* w;             // row width
    const int* stream;
    const uint8_t* low;       // rows of a lowpass component (raw in a K-frame)
    int ntiles;
};
constexpr int RLE_THREADS = 256, RLE_PER_THREAD = 8, RLE_CHUNK = RLE_THREADS * RLE_PER_THREAD, RLE_TILE = 4096;

struct CompTable {
    const int* tile0;         // first RLE tile of the component (global)
    const uint8_t* low;
    const int* stream;
    const long long* elem;    // element offset of the component inside its stream
    const uint8_t* level;     // 0 lowpass, j = pyramid level j (1 finest)
    const uint8_t* plane;     // 0 Y, 1 Co, 2 Cg
    const uint8_t* ey;        // one element stands for 2^ey x 2^ex luma samples
    const uint8_t* ex;
    int ncomp;
};

// element-wise kernels: ELEM_THREADS threads, ELEM_PER_THREAD elements each
constexpr int ELEM_THREADS = 256, ELEM_PER_THREAD = 8, ELEM_BLOCK = ELEM_THREADS * ELEM_PER_THREAD;

// first and last kernel of every step: the call records' coder-state fields from
// the device-resident state, and the outcome of the call (statuses, lengths,
// frame types; the state advanced where the call succeeded); a thread per stream
__global__ void k_step_begin(const SDesc* sd, SCall* sc, SCtl* ctl, int n);
__global__ void k_step_commit(const SDesc* sd, const SCall* sc, SResult* rs, SCtl* ctl, int n);
__global__ void k_colour_fwd_b(const SDesc* sd, const SCall* sc, const int* blk_stream, float* planes,
                               uint8_t* luma0, uint8_t* luma1);
// motion search of the P-frames of streams with a motion range: one block per 16 x 16 luma block,
// any multiple of 32 threads up to 1024 walking the (2W + 1)^2 candidates; dynamic shared memory of
// (16 + 2 W_max) * ws bytes, ws = 16 + 2 W_max + 4 rounded up to a multiple of 4 (W_max the largest
// range of the launch)
__global__ void k_motion_b(const SDesc* sd, const SCall* sc, const int* blk_stream, const uint8_t* luma0,
                           const uint8_t* luma1, int8_t* mv, int ws);
// residuals of motion-compensated P-frames (after k_quant_b wrote their codes)
__global__ void k_mc_resid_b(const int16_t* est0, const int16_t* est1, RowTable rt, CompTable ct,
                             const SDesc* sd, const SCall* sc, const int8_t* mv, int16_t* res);
// decoder: codes and coefficients of motion-compensated P-frames
__global__ void k_mc_recon_b(const int16_t* res, int16_t* dst0, int16_t* dst1, RowTable rt, CompTable ct,
                             const SDesc* sd, const SCall* sc, const SResult* rs, float* coef);
__global__ void k_colour_inv_b(const ScaleDesc* sdesc, const SCall* sc, const SResult* rs, const int* blk_stream,
                               const float* rplanes, const float* dcoef);
// k_quant_b<POW2> over nblocks element blocks; pow2: every stream's steps are powers of two
// (the quotients are products; the kernel carries no division code)
void launch_quant_b(bool pow2, int nblocks, cudaStream_t st, const float* coef, int16_t* est0, int16_t* est1,
                    const PDesc* pd, const int* blk_plane, const SDesc* sd, const SCall* sc, int16_t* res,
                    SResult* out);
__global__ void k_unquant_b(const int16_t* res, int16_t* dst0, int16_t* dst1, const PDesc* pd, const int* blk_plane,
                            const SDesc* sd, const SCall* sc, const SResult* rs, float* coef);
__global__ void k_unquant_keylow_b(const int16_t* res, int16_t* dst0, int16_t* dst1, const PDesc* pd, int nplanes,
                                   const SDesc* sd, const SCall* sc, const SResult* rs, float* coef);
// RLE: one block of RLE_THREADS per tile; token counts, then (after their
// exclusive scan) the tokens; the header writes the component counts
__global__ void k_rle_count_b(const int16_t* res, RleTiles tt, const SCall* sc, uint32_t* cnt);
__global__ void k_rle_write_b(const int16_t* res, RleTiles tt, const SDesc* sd, const SCall* sc,
                              const uint32_t* tileoff, SResult* out);
__global__ void k_stream_header_b(const SDesc* sd, const SCall* sc, const uint32_t* tileoff, CompTable ct,
                                  const int8_t* mv, SResult* out);
__global__ void k_dec_parse_b(const SDesc* sd, const SCall* sc, const SResult* enc, CompTable ct,
                              uint32_t* comp_tok, SResult* out);
__global__ void k_dec_base_b(const SDesc* sd, int nstreams, const SResult* rs, uint32_t* tok_base, uint32_t* tile_base);
// the decoder's token tiles: DEC_TILE tokens of one stream each, DEC_THREADS threads of
// DEC_PER_THREAD consecutive tokens; grid-stride loops over the call's tiles
constexpr int DEC_THREADS = 256, DEC_PER_THREAD = 8, DEC_TILE = DEC_THREADS * DEC_PER_THREAD;
constexpr int DEC_MAX_COMP = 3 * (1 + CVC_MAX_LEVELS * 64);   // components of a stream, at most
__global__ void k_dec_count_b(const SDesc* sd, const SCall* sc, const SResult* rs, const uint32_t* tile_base,
                              int nstreams, const uint32_t* comp_tok, CompTable ct, uint32_t* tile_sum, SResult* out);
__global__ void k_dec_scatter_b(const SDesc* sd, const SCall* sc, const SResult* rs, const uint32_t* tile_base,
                                int nstreams, const uint32_t* comp_tok, CompTable ct, const uint32_t* tile_pre,
                                uint32_t* comp_codes, int16_t* res);
__global__ void k_dec_check_b(const SDesc* sd, const SResult* rs, const uint32_t* comp_codes, CompTable ct,
                              SResult* out);

// exclusive scan of n values into out[0..n] (out[n] = total); tmp holds
// ceil(n / 2048) + 1 values.
cudaError_t exclusive_scan(const uint32_t* in, uint32_t n, uint32_t* out, uint32_t* tmp, cudaStream_t st);
// the same with n read from device memory (*d_n <= n_max); a fixed grid, so
// the launch sequence does not depend on host-side sizes
cudaError_t exclusive_scan_dev(const uint32_t* in, const uint32_t* d_n, uint32_t n_max, uint32_t* out, uint32_t* tmp,
                               cudaStream_t st);

}  // namespace cvc
