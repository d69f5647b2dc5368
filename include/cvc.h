/*
 * cvc.h -- C ABI of the B300 contourlet video codec library (libcvc.so).
 *
 * The library implements the data-parallel hot path of CVC, the contourlet
 * video codec of Katsigiannis, Papaioannou and Maroulis (arXiv:1510.00561):
 * colour conversion and chroma subsampling (§3.1), the contourlet transform
 * (§2.1, §3.3), lowpass normalisation (§3.4), quantisation and rounding
 * (§3.5, §3.6), K/P frame differencing (§3.7) and run-length coding (§3.8),
 * and the inverse chain of the decoder.  Every step runs in CUDA kernels
 * written for sm_103a; there is no CPU fallback.
 *
 * Conventions for every call below:
 *   - Pointers named d_* are DEVICE pointers owned by the caller; the library
 *     never frees them and only touches them on the given stream.
 *   - Calls are asynchronous on `stream` unless they return a host value that
 *     needs the GPU's result (out_len / frame_type of cvc_encode_frame, the
 *     status of cvc_decode_frame); those synchronise the stream before
 *     returning.
 *   - A call that fails leaves the codec state (key-frame state, frame
 *     counter) exactly as it was.
 *   - A context (cvc_codec, cvc_ct_plan) is not thread-safe; distinct
 *     contexts are independent and may run concurrently on distinct streams.
 *   - CUDA errors map to CVC_ERR_CUDA; allocation failures to CVC_ERR_NOMEM.
 */
#ifndef CVC_H
#define CVC_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    CVC_OK = 0,
    CVC_ERR_INVALID_ARG = 1,  /* argument outside its documented range            */
    CVC_ERR_UNSUPPORTED = 2,  /* valid but not supported by this build            */
    CVC_ERR_CAPACITY = 3,     /* output buffer too small; *out_len = bytes needed */
    CVC_ERR_OVERFLOW = 4,     /* a quantised code left the int16 range            */
    CVC_ERR_CORRUPT = 5,      /* malformed or mismatched bitstream                */
    CVC_ERR_CUDA = 6,         /* a CUDA runtime call failed                       */
    CVC_ERR_TIMEOUT = 7,      /* a bounded device wait gave up                    */
    CVC_ERR_NOMEM = 8,        /* device or host allocation failed                 */
    CVC_ERR_STATE = 9         /* P-frame without its reference frame              */
} cvc_status;

/* a CUDA stream handle (the same type as cudaStream_t); NULL = legacy stream */
typedef struct CUstream_st* cvc_stream_t;

#define CVC_MAX_LEVELS 6
#define CVC_MAX_DIRS_LOG2 6
#define CVC_MAX_SUBBANDS (1 + CVC_MAX_LEVELS * 64)

/* Human-readable name of a status code (static string). */
const char* cvc_status_string(cvc_status s);

/* ------------------------------------------------------------------ layout
 * Coefficient layout of one plane (§3.3: the coarsest lowpass image plus
 * the directional subbands of each scale), float elements, row-major
 * subbands packed back to back:
 *   [lowpass (h>>L) x (w>>L)] [level 1 (finest): 2^k1 subbands] ... [level L]
 * Level j works on the (h>>(j-1)) x (w>>(j-1)) detail image; with k = k_j:
 *   k = 0: one subband, the detail itself
 *   k = 1: two quincunx halves, each (hj) x (wj/2), row-compacted
 *   k >= 2: subbands 0 .. 2^(k-1)-1 are (hj>>(k-1)) x (wj/2) (wedges about the
 *          horizontal-frequency axis), the rest (hj/2) x (wj>>(k-1)).
 * Directions are in filter-bank tree order (wedge slope increasing within
 * each half).  `kind`: 0 lowpass, 1 / 2 the two wedge families, 3 undivided
 * detail, 4 quincunx half.
 * Plane sizes must be multiples of cvc_modulus(levels, dirs_log2).          */
typedef struct {
    long long off;
    int h, w, level, dir, kind;
} cvc_subband;

typedef struct {
    int height, width, levels, dirs_log2[CVC_MAX_LEVELS];
    int modulus;
    int nsub;                             /* lowpass + directional subbands */
    cvc_subband sub[CVC_MAX_SUBBANDS];
    long long total;                      /* coefficients of one plane      */
} cvc_ct_layout_t;

/* Smallest size every plane dimension must be a multiple of:
 * max(2^L, max_j 2^(j-1) * max(2^(k_j-1), 2)).  Returns 0 for bad arguments. */
int cvc_modulus(int levels, const int* dirs_log2);

/* Fill *out for an h x w plane.  INVALID_ARG unless 1 <= levels <= 6,
 * 0 <= dirs_log2[j] <= 6 and h, w are positive multiples of the modulus.    */
cvc_status cvc_ct_layout(int h, int w, int levels, const int* dirs_log2, cvc_ct_layout_t* out);

/* ------------------------------------------------- contourlet transform
 * §2.1: Laplacian pyramid with the CDF 9/7 pair (periodic extension) whose
 * detail images feed directional filter banks of ladder fan filters.
 * A plan fixes the plane size, the decomposition and a batch count, and
 * owns the device workspace (about 1.7 plane sizes per batch entry).
 * Data layout: d_x is `batch` dense planes of h x w floats (row-major,
 * plane stride h*w); d_coeffs is `batch` coefficient vectors of
 * layout.total floats.  The four maps are linear:
 *   forward A: x -> coeffs;  inverse S: coeffs -> x  (S A = identity);
 *   forward_adjoint A^T: coeffs -> x;  inverse_adjoint S^T: x -> coeffs.
 * Input and output buffers must not overlap.                               */
typedef struct cvc_ct_plan cvc_ct_plan;

cvc_status cvc_ct_plan_create(int h, int w, int levels, const int* dirs_log2, int batch,
                              cvc_ct_plan** out);
/* the same with a DFB prototype of dfb_taps (4, 6 or 8; see cvc_params)   */
cvc_status cvc_ct_plan_create_taps(int h, int w, int levels, const int* dirs_log2, int batch, int dfb_taps,
                                   cvc_ct_plan** out);
cvc_status cvc_ct_plan_destroy(cvc_ct_plan* plan);
/* Fusion depth of the forward transform and the inverse (see
 * cvc_batch_set_fusion): the most coarse levels of each plane run in one
 * block with their images in shared memory; changes no result.  Waits for
 * the device, rebuilds the plan's tables.  Errors: INVALID_ARG, NOMEM.     */
cvc_status cvc_ct_plan_set_fusion(cvc_ct_plan* plan, int levels);
/* total coefficients of one plane of this plan (layout.total) */
long long cvc_ct_plan_coeffs(const cvc_ct_plan* plan);

cvc_status cvc_ct_forward(cvc_ct_plan* plan, const float* d_x, float* d_coeffs, cvc_stream_t stream);
cvc_status cvc_ct_inverse(cvc_ct_plan* plan, const float* d_coeffs, float* d_x, cvc_stream_t stream);
cvc_status cvc_ct_forward_adjoint(cvc_ct_plan* plan, const float* d_coeffs_bar, float* d_x_bar,
                                  cvc_stream_t stream);
cvc_status cvc_ct_inverse_adjoint(cvc_ct_plan* plan, const float* d_x_bar, float* d_coeffs_bar,
                                  cvc_stream_t stream);

/* Soft thresholding of a plan's coefficients with one threshold per
 * directional subband, for gradient-based tuning of the thresholds (a
 * differentiable stand-in for the hard subband threshold of §3.5):
 *   y = sign(c) * max(|c| - T[s], 0) in directional subband s (layout order,
 *   s = 0 .. cvc_ct_plan_subbands - 1, shared by every batch entry); the
 *   lowpass is copied unchanged.
 * The backward pass takes dL/dy and returns
 *   dL/dc = dL/dy * [|c| > T[s]] (lowpass: dL/dy) and
 *   dL/dT[s] = -sum over subband s of every batch entry of dL/dy * sign(c) * [|c| > T[s]],
 * the latter summed in a fixed order (repeatable bit for bit).
 * d_thresholds and d_grad_thresholds hold cvc_ct_plan_subbands floats;
 * coefficient buffers are `batch` vectors of layout.total floats.  d_out may
 * equal d_coeffs and d_grad_coeffs may equal d_grad_out; no other overlap.
 * Asynchronous on `stream`.  Errors: INVALID_ARG, CUDA.                    */
int cvc_ct_plan_subbands(const cvc_ct_plan* plan);
cvc_status cvc_ct_soft_threshold(cvc_ct_plan* plan, const float* d_coeffs, const float* d_thresholds,
                                 float* d_out, cvc_stream_t stream);
cvc_status cvc_ct_soft_threshold_backward(cvc_ct_plan* plan, const float* d_coeffs, const float* d_thresholds,
                                          const float* d_grad_out, float* d_grad_coeffs,
                                          float* d_grad_thresholds, cvc_stream_t stream);

/* ---------------------------------------------------------------- codec
 * One video stream: encoder and decoder state resident on the device.
 *   width, height   frame size in pixels, 1..65535 (padded internally to the
 *                   modulus by half-sample mirroring; chroma is 4:2:0)
 *   levels          LP levels, 1..6 (§3.3)
 *   dirs_log2[j]    DFB stages of level j+1 (finest first), 0..6
 *   qph, qpl        quantisation steps of subbands [1,181] and lowpass [1,71] (§3.5)
 *   subband_threshold  subband coefficients with |c| below it become 0 (>= 0)
 *   key_interval    frame i (since create/reset) is a K-frame iff i % key_interval == 0 (§3.7)
 *   chroma_420      must be 1
 *   motion_range    W in 0..CVC_MAX_MOTION_RANGE.  0: P-frames predict every
 *                   component from the previous frame's codes at the same
 *                   position (type byte 1).  W > 0 (§3.2, §3.7): full-search
 *                   block matching of each 16x16 block of the padded luma
 *                   plane against the previous frame's, over every
 *                   displacement in [-W, W]^2 that keeps the block inside the
 *                   plane, by smallest sum of squared differences (ties: the
 *                   smaller |dy| + |dx|, then the first in raster order, dy
 *                   then dx ascending); P-frames (type byte 2) then carry one
 *                   int8 (dy, dx) per block, raster order, after their tokens,
 *                   and each component is predicted through the vector of the
 *                   block under each element: an element standing for 2^ey x
 *                   2^ex luma samples (its plane's size over the component's,
 *                   doubled for chroma) uses the block of luma sample
 *                   (i 2^ey, j 2^ex) (the last block row / column past the
 *                   plane) and reads the previous code at (i + dy/2^ey,
 *                   j + dx/2^ex), each quotient rounded half away from zero,
 *                   clamped to the component.
 *   storage8        0: lossless YCoCg-R colour and int16 codes.  1: the
 *                   paper's 8-bit storage (§3.1, §3.6): the colour
 *                   transform of Table I in its real-valued form, every
 *                   component rounded (ties away from zero) to a byte,
 *                   chroma offset by +127 and clamped to [0, 255] (the
 *                   decoder subtracts 127); every code (the quotient by
 *                   QPH / QPL, rounded) is clamped to a byte: subbands
 *                   [-128, 127], the normalised lowpass [0, 255].
 *                   Header byte 5 bit 0 records it; a decoder refuses a
 *                   stream of the other storage.
 *   dfb_taps        length of the DFB ladder's half-band prototype (§2.1
 *                   fixes none): 0 or 4, (-1, 9, 9, -1)/16, run by the
 *                   tiled DFB kernels; 6 or 8, the longer Lagrange
 *                   half-band interpolators (3, -25, 150, 150, -25, 3)/256
 *                   and (-5, 49, -245, 1225, 1225, -245, 49, -5)/2048, a
 *                   sharper directional split, run by the same kernels with
 *                   wider halos.  Header byte 5 bits 1-2 record it (0, 1, 2). */
#define CVC_MAX_MOTION_RANGE 64
typedef struct {
    int width, height;
    int levels;
    int dirs_log2[CVC_MAX_LEVELS];
    int qph, qpl;
    float subband_threshold;
    int key_interval;
    int chroma_420;
    int motion_range;
    int storage8;
    int dfb_taps;
} cvc_params;

typedef struct {
    int padded_height, padded_width;           /* luma plane as transformed        */
    int chroma_height, chroma_width;           /* unpadded 4:2:0 chroma size       */
    int padded_chroma_height, padded_chroma_width;
    long long coeffs;                          /* coefficients of one frame (Y,Co,Cg) */
    int components;                            /* bitstream components per frame   */
    long long max_stream_bytes;                /* worst-case encoded frame size     */
} cvc_codec_info_t;

typedef struct cvc_codec cvc_codec;

cvc_status cvc_create(const cvc_params* params, cvc_codec** out);
cvc_status cvc_destroy(cvc_codec* codec);
/* Next encoded frame is a K-frame; the decoder expects a K-frame next.  The
 * reset travels with the codec's next call (it takes effect in stream order,
 * after calls already queued); no device call is made here.                */
cvc_status cvc_reset(cvc_codec* codec);
cvc_status cvc_codec_info(const cvc_codec* codec, cvc_codec_info_t* out);

/* Encode one frame.
 *   d_rgb        height rows of width*3 interleaved R,G,B bytes, row pitch pitch_bytes
 *   d_out        receives the frame bitstream (device), capacity out_cap bytes
 *   *out_len     (host) bytes written; on CVC_ERR_CAPACITY the bytes needed
 *   *frame_type  (host, may be NULL) 0 = K-frame, 1 = P-frame
 * Bitstream (little-endian): 32-byte header {"CVC1", u8 version=1, u8
 * flags (bit 0 storage8, bits 1-2 dfb_taps / 2 - 2), u8 type, u8 levels, u32 frame index, u16 height, u16 width, u8
 * dirs_log2[6], u16 qph, u16 qpl, u16 0, u32 ncomp}, then ncomp u32 token
 * counts, then the
 * int16 tokens of every component.  Components run Y, Co, Cg, each in the
 * coefficient layout order.  The K-frame lowpass holds its column-differenced
 * codes raw; every other component holds, row by row, one token per non-zero
 * code and the pair (0, n) per maximal run of n zeros (§3.8).
 * Synchronises `stream`.  Errors: INVALID_ARG, CAPACITY, OVERFLOW, CUDA.    */
cvc_status cvc_encode_frame(cvc_codec* codec, const uint8_t* d_rgb, size_t pitch_bytes,
                            uint8_t* d_out, size_t out_cap, size_t* out_len, int* frame_type,
                            cvc_stream_t stream);

/* Decode one frame produced by cvc_encode_frame of a codec with the same
 * parameters into d_rgb (height rows of width*3 bytes, row pitch pitch_bytes).
 * Synchronises `stream`.  Errors: INVALID_ARG, CORRUPT (malformed stream or
 * parameter mismatch), STATE (P-frame that does not follow the last decoded
 * frame), CUDA.                                                             */
cvc_status cvc_decode_frame(cvc_codec* codec, const uint8_t* d_in, size_t in_len, uint8_t* d_rgb,
                            size_t pitch_bytes, cvc_stream_t stream);

/* Scalable decoding (§3.3: each LP scale of a frame can be decoded on its
 * own).  As cvc_decode_frame, but the output is the frame at pyramid scale
 * `scale` (0 <= scale <= levels): ceil(height / 2^scale) rows of
 * ceil(width / 2^scale) * 3 bytes at row pitch pitch_bytes.  Scale s
 * inverts only the lowpass and levels s+1..L of each plane, i.e. the
 * coefficients of its level-s lowpass image under an (L - s)-level
 * transform, and divides the result by the DC gain 2^s of s levels; scale L
 * shows the lowpass band itself.  The whole bitstream is still parsed and
 * the decoder state (the P-frame reference) updated in full, so the scale
 * may change from frame to frame, and a later full-scale decode is the same
 * as if every frame had been decoded at full scale.  Scale 0 is
 * cvc_decode_frame.  Errors: as cvc_decode_frame; INVALID_ARG also for a
 * scale outside [0, levels].                                                */
cvc_status cvc_decode_frame_scaled(cvc_codec* codec, const uint8_t* d_in, size_t in_len, int scale,
                                   uint8_t* d_rgb, size_t pitch_bytes, cvc_stream_t stream);

/* Asynchronous encode and decode.  The paper's encoder keeps a frame on the
 * GPU from the colour conversion to the frame-type step (§3.7, §3.10);
 * these forms keep the whole call there: nothing waits on the host, the
 * outcome goes to DEVICE memory, and the coder state (frame index, K/P
 * schedule, the decoder's reference) lives and advances on the device, so
 * calls queue back to back on `stream` and give exactly the bytes and
 * pixels of the synchronous calls made in the same order.
 *   cvc_encode_frame_async: as cvc_encode_frame; the step writes the
 *     encoded length (the length needed when out_cap is too small) to
 *     *d_out_len, the frame type (0 K, 1 P, 2 P with motion) to
 *     *d_frame_type and the call's status (OK, CAPACITY, OVERFLOW) to
 *     *d_status; each pointer is device memory and may be NULL.
 *   cvc_decode_frame_async: as cvc_decode_frame_scaled; d_in holds in_cap
 *     bytes, and the frame's length is *d_in_len (device memory, read when
 *     the step runs, at most in_cap; NULL: in_cap is the length), e.g. the
 *     d_out_len of an encode queued before it.  The status (OK, CORRUPT,
 *     STATE) goes to *d_status (device, may be NULL).
 * A failed call leaves the coder state unchanged, as the synchronous forms
 * do; the first failure since the last cvc_get_error is also kept in the
 * codec's device status word.  Argument checks that need no device data
 * happen on the host (INVALID_ARG: nothing queued); the call returns CUDA
 * if queueing failed, otherwise OK.  The host may run up to 8 calls ahead
 * of the device; a ninth waits for the first of them to finish.  Stage
 * timing (cvc_codec_set_timing) counts synchronous calls only.  Buffers
 * must stay valid until the stream has run the call.                        */
cvc_status cvc_encode_frame_async(cvc_codec* codec, const uint8_t* d_rgb, size_t pitch_bytes, uint8_t* d_out,
                                  size_t out_cap, size_t* d_out_len, int* d_frame_type, cvc_status* d_status,
                                  cvc_stream_t stream);
cvc_status cvc_decode_frame_async(cvc_codec* codec, const uint8_t* d_in, size_t in_cap, const size_t* d_in_len,
                                  int scale, uint8_t* d_rgb, size_t pitch_bytes, cvc_status* d_status,
                                  cvc_stream_t stream);
/* The codec's device status word: the first non-OK status of an
 * asynchronous call since the last read (CVC_OK if none), read and cleared
 * in `stream` order (calls queued on `stream` before this one are seen).
 * Synchronises `stream`.  Errors: INVALID_ARG, CUDA.                        */
cvc_status cvc_get_error(cvc_codec* codec, cvc_stream_t stream, cvc_status* status);

/* Transmission-side scalability (§3.3: a receiver's resolution is served by
 * dropping what refers to higher resolutions, without re-encoding).  Copies
 * the frame `in` (HOST memory, in_len bytes, from a codec with `params`)
 * into `out` (HOST memory) without the components of its finest `drop`
 * levels: their token counts become 0, their tokens are left out, and
 * header bytes 26-27 (0 in a complete frame) hold `drop`; the motion
 * vectors of a P-frame with motion stay after the tokens.  A deflated frame
 * (version byte 2, cvc_deflate_frame) loses the DEFLATE streams and segment
 * entries of those components the same way (its stream lengths become 0),
 * and is byte-identical to deflating the frame with the levels dropped.  A
 * CVC-NTS frame (version byte 3, one stream) has nothing to drop:
 * UNSUPPORTED.  A frame that already left out d0 levels can only lose more
 * (drop >= d0).  `out` may be
 * `in` (the tokens only move forward).  Host work only, no device call.
 * A decoder accepts such a frame at scales >= drop (cvc_decode_frame_scaled;
 * STATE below that).  Afterwards the decoder state of levels 1..drop is
 * missing: a P-frame then decodes only at scales >= the largest drop since
 * the last K-frame (STATE otherwise), and a K-frame resets that floor to its
 * own drop.  Errors: INVALID_ARG (bad params, drop outside [d0, levels]),
 * CORRUPT (not a frame of these params), CAPACITY (*out_len = bytes needed),
 * UNSUPPORTED.                                                               */
cvc_status cvc_stream_drop_levels(const cvc_params* params, const uint8_t* in, size_t in_len, int drop,
                                  uint8_t* out, size_t out_cap, size_t* out_len);

/* Inspection of the last encode / decode (for parity checks): copies into
 * d_out (device, at least cap_elems floats)
 *   which = 0: the encoder's padded float planes Y, Co, Cg (before the transform)
 *   which = 1: the encoder's transform coefficients (Y, Co, Cg layouts back to back)
 *   which = 2: the decoder's reconstructed padded planes Y, Co, Cg (before rounding)
 * Asynchronous on `stream`.  INVALID_ARG if cap_elems is too small.          */
cvc_status cvc_codec_inspect(const cvc_codec* codec, int which, float* d_out, size_t cap_elems,
                             cvc_stream_t stream);

/* --------------------------------------------------------------- DEFLATE
 * The last stage of CVC (§3.9), in its scalable mode: the tokens of every
 * component become a raw DEFLATE stream (RFC 1951) of their own, so that any
 * subset of components can be sent or dropped.  Each stream is one final
 * block with dynamic Huffman codes (at most 15 bits) over the token bytes
 * taken as literals, without LZ77 matches, which lets both directions run
 * as data-parallel kernels.  Container ("deflated frame"): the 32-byte CVC
 * header with version byte 2, the ncomp u32 token counts, ncomp u32 stream
 * byte lengths (0 for a component without tokens), for every 256-byte
 * segment of every component's token bytes (in component order) the u16 bit
 * length of its literals, zero padding to 4 bytes, the streams back to back
 * (each byte-aligned, its header, literals and end-of-block code), then the
 * motion vectors of a type-2 frame.  Any inflater decodes each stream alone;
 * the segment lengths are the entry points of the parallel inflate.
 * CVC-NTS ("non transmission scalable", §3.9; cvc_deflate_set_nts): the
 * token bytes of the whole frame, in component order, become ONE stream.
 * Its container has version byte 3 and one u32 stream length in place of
 * the ncomp of them, and its 256-byte segments run over the whole token
 * bytes; the rest is as above.  Levels can no longer be dropped in transit,
 * but the inflated frame still decodes at any scale.
 * A context holds device scratch for up to max_frames frames of one
 * parameter set (cvc_deflate_create: 1); a call covers any number of frames
 * up to it in one launch sequence.                                         */
typedef struct cvc_deflate_ctx cvc_deflate_ctx;
cvc_status cvc_deflate_create(const cvc_params* params, cvc_deflate_ctx** out);
cvc_status cvc_deflate_create_batch(const cvc_params* params, int max_frames, cvc_deflate_ctx** out);
cvc_status cvc_deflate_destroy(cvc_deflate_ctx* ctx);
/* on != 0: later deflate calls write CVC-NTS containers (version 3), 0:
 * scalable ones (version 2, the default).  Inflate reads either.
 * Errors: INVALID_ARG (ctx NULL).                                           */
cvc_status cvc_deflate_set_nts(cvc_deflate_ctx* ctx, int on);
/* d_in: one frame of cvc_encode_frame (version byte 1, possibly without some
 * levels, cvc_stream_drop_levels) in device memory; d_out (device, 4-byte
 * aligned, out_cap bytes) receives the deflated frame; *out_len (host) its
 * length, or the bytes needed on CAPACITY.  Synchronises `stream`.
 * Errors: INVALID_ARG, CORRUPT, CAPACITY, CUDA.                              */
cvc_status cvc_deflate_frame(cvc_deflate_ctx* ctx, const uint8_t* d_in, size_t in_len, uint8_t* d_out,
                             size_t out_cap, size_t* out_len, cvc_stream_t stream);
/* the inverse: a deflated frame of this context's parameters back to the
 * frame cvc_decode_frame reads (device memory both), from either container
 * form.  CORRUPT for anything but the containers above (a stream must decode to exactly its token bytes,
 * each segment to its recorded bit length, and end with the end-of-block
 * code).  Synchronises `stream`.                                            */
cvc_status cvc_inflate_frame(cvc_deflate_ctx* ctx, const uint8_t* d_in, size_t in_len, uint8_t* d_out,
                             size_t out_cap, size_t* out_len, cvc_stream_t stream);
/* the same for n frames at once (n <= the context's max_frames): the pointer
 * and size arrays are HOST arrays of n entries (the buffers they point to
 * are device memory); out_len[i] and status[i] (may be NULL) are per frame.
 * Returns INVALID_ARG or CUDA for the call, else the first non-OK status.  */
cvc_status cvc_deflate_frames(cvc_deflate_ctx* ctx, int n, const uint8_t* const* d_in, const size_t* in_len,
                              uint8_t* const* d_out, const size_t* out_cap, size_t* out_len, cvc_status* status,
                              cvc_stream_t stream);
cvc_status cvc_inflate_frames(cvc_deflate_ctx* ctx, int n, const uint8_t* const* d_in, const size_t* in_len,
                              uint8_t* const* d_out, const size_t* out_cap, size_t* out_len, cvc_status* status,
                              cvc_stream_t stream);

/* --------------------------------------------------------------- batches
 * Many independent streams, each with its own cvc_params (any mix of frame
 * sizes and decompositions), coded together: every kernel of a step covers
 * all streams of the batch (its blocks find their stream through tables
 * built at creation), and the step's fixed launch sequence is captured once
 * per step kind in a CUDA graph and replayed, so a step costs one graph
 * launch, two small copies and one synchronisation whatever the number of
 * streams.  Each stream's bitstream, reconstruction and coder state are
 * bit-identical to those of a cvc_codec with the same parameters fed the
 * same frames; a stream that takes no part in a step is left untouched.    */
typedef struct cvc_batch cvc_batch;

#define CVC_STEP_ENCODE 1
#define CVC_STEP_DECODE 2
#define CVC_STEP_ENCODE_DECODE 3   /* encode, then decode this step's own output */

typedef struct {
    const uint8_t* d_rgb;   /* encoder input as in cvc_encode_frame; NULL: the stream does not encode */
    size_t pitch_bytes;
    uint8_t* d_out;         /* encoder output, 4-byte aligned, out_cap bytes */
    size_t out_cap;
    const uint8_t* d_in;    /* decoder input; ignored when the same step encodes the stream
                               (CVC_STEP_ENCODE_DECODE): the decoder then reads d_out */
    size_t in_len;
    uint8_t* d_rgb_out;     /* decoder output as in cvc_decode_frame; NULL: the stream does not decode */
    size_t pitch_out;
} cvc_batch_io;

typedef struct {
    cvc_status enc_status;  /* as cvc_encode_frame (CVC_OK when the stream did not encode) */
    cvc_status dec_status;  /* as cvc_decode_frame (CVC_OK when the stream did not decode) */
    size_t out_len;         /* as cvc_encode_frame's *out_len; 0 when the stream did not encode */
    int frame_type;         /* encoded frame: 0 K, 1 P, -1 none */
    int dec_frame_type;     /* decoded frame: 0 K, 1 P, -1 none or rejected */
    uint32_t dec_frame_index;
} cvc_batch_result;

/* n >= 1 streams with params[0..n-1].  Errors: INVALID_ARG, UNSUPPORTED
 * (as cvc_create, or a batch whose token space exceeds 32 bits), NOMEM, CUDA. */
cvc_status cvc_batch_create(const cvc_params* params, int n, cvc_batch** out);
cvc_status cvc_batch_destroy(cvc_batch* batch);
/* Device bytes cvc_batch_create would allocate for these streams (host-only,
 * no device call): the basis of admission against a memory budget.         */
cvc_status cvc_batch_device_bytes(const cvc_params* params, int n, size_t* bytes);
cvc_status cvc_batch_info(const cvc_batch* batch, int i, cvc_codec_info_t* out);
/* as cvc_reset for stream i (i < 0: every stream) */
cvc_status cvc_batch_reset(cvc_batch* batch, int i);

/* One step of kind `what` (CVC_STEP_*) over every stream: io[i] and res[i]
 * belong to stream i.  Synchronises `stream`.  Returns INVALID_ARG (nothing
 * was done) or CUDA for the call; otherwise the first non-OK status in res
 * (stream order, encoder before decoder), or CVC_OK.                        */
cvc_status cvc_batch_step(cvc_batch* batch, int what, const cvc_batch_io* io, cvc_batch_result* res,
                          cvc_stream_t stream);

/* The same with every decoding stream of the step output at pyramid scale
 * `scale` (as cvc_decode_frame_scaled; each d_rgb_out sized for that scale).
 * INVALID_ARG if a decoding stream has fewer than `scale` levels.  Each
 * scale replays its own captured graph.                                     */
cvc_status cvc_batch_step_scaled(cvc_batch* batch, int what, const cvc_batch_io* io, int scale,
                                 cvc_batch_result* res, cvc_stream_t stream);

/* The asynchronous batch step (see cvc_encode_frame_async): io as for
 * cvc_batch_step_scaled (host array, checked on the host); d_in_len, if not
 * NULL, is a DEVICE array of n decoder input lengths read when the step
 * runs (each at most io[i].in_len, the buffer's capacity); d_res, if not
 * NULL, a DEVICE array of n results that the step writes.  Every stream's
 * coder state advances on the device where its call succeeded; the first
 * failure of a stream is kept in its device status word
 * (cvc_batch_get_error).  Returns INVALID_ARG (nothing queued), CUDA, or OK. */
cvc_status cvc_batch_step_async(cvc_batch* batch, int what, const cvc_batch_io* io, const size_t* d_in_len,
                                int scale, cvc_batch_result* d_res, cvc_stream_t stream);
/* as cvc_get_error for stream i of a batch */
cvc_status cvc_batch_get_error(cvc_batch* batch, int i, cvc_stream_t stream, cvc_status* status);

/* Launch shapes (they change no result): rows per block of the row kernels
 * of motion-compensated frames, one warp per row (1..32; `rle_rows` names it
 * for the row kernels it once set), and blocks of the decoder's grid-stride
 * token-tile kernels (1..65535).
 * Fusion depth (changes no result either): the most coarse pyramid levels of
 * each plane that run in its pyramid tail, one block per plane with the
 * levels' images resident in shared memory (§2.1: the LP iterated on the
 * lowpass, a DFB on every detail); a plane's tail takes as many of them as
 * fit 227 KB of shared memory (1080p: luma level 5, chroma levels 4-5; QCIF:
 * luma levels 2-3, the whole chroma planes); 0 runs every level as its own
 * launches, the default (one block per plane runs the coarse levels' tiles
 * one after the other, which on a 1080p frame is slower than their own
 * launches; the autotuner tries tails of 1, 2 and CVC_MAX_LEVELS levels).
 * Row-split DFB block width (changes no result either): threads per block of
 * the launches of DFB stages 3 and later (§2.1), 128 (four warps, each a run
 * of the tile's rows) or 256 (eight warps, shorter runs: sooner done where a
 * launch has fewer blocks than the GPU holds); 0, the default, takes 256 for
 * a launch of less than a wave of 128-thread blocks, else 128.  Anything
 * else is INVALID_ARG.
 * cvc_batch_autotune times candidate shapes, fusion depths and block widths
 * on steps over `io` (the outputs of io are written; no coder state
 * changes), keeps the fastest and returns it in shape[4] = {rle_rows,
 * tok_blocks, fusion depth, row-split block width} (may be NULL).  Graph
 * replay can be switched off (on = 0) to run the same launches one by one. */
cvc_status cvc_batch_set_shape(cvc_batch* batch, int rle_rows, int tok_blocks);
cvc_status cvc_batch_set_fusion(cvc_batch* batch, int levels);
cvc_status cvc_batch_set_dfb_threads(cvc_batch* batch, int threads);
cvc_status cvc_batch_autotune(cvc_batch* batch, int what, const cvc_batch_io* io, int reps, int* shape,
                              cvc_stream_t stream);
cvc_status cvc_batch_set_graphs(cvc_batch* batch, int on);
/* Stage timing of a batch, as cvc_codec_set_timing / cvc_codec_timing (each
 * stage's events bracket that stage's launches over all streams).  While
 * timing is on, steps run as direct launches instead of graph replays.     */
cvc_status cvc_batch_set_timing(cvc_batch* batch, int on);
cvc_status cvc_batch_timing(const cvc_batch* batch, double* ms, long long* launches);

/* ---------------------------------------------------------------- server
 * A continuous-batching request loop over many concurrent streams (the
 * deployment form of the codec for conferencing: §4's real-time claim, many
 * streams per GPU).  Streams ("sessions") open and close at any time;
 * frames are submitted as they arrive and complete asynchronously.
 *   - Admission by memory: a session is admitted when a slot for its
 *     parameters is free or a new shard fits the budget (the exact device
 *     bytes of cvc_batch_device_bytes); until then it waits (first fit, in
 *     opening order) and its submitted frames queue.
 *   - Shards: sessions with identical parameters share a shard of
 *     slots_per_shard slots; one step of a shard codes the next queued
 *     request of each of its sessions (one CUDA-graph launch).  Every shard
 *     runs on its own CUDA stream, so shards overlap on the device; requests
 *     that arrive while a shard's steps run go into its next step, which is
 *     queued at once when steps_in_flight allows it.
 *   - Coder state stays resident in the shard; a session's requests run in
 *     submission order.  Each result is bit-identical to a cvc_codec of the
 *     same parameters fed the same requests, whatever else is in flight.
 *   - An empty shard is freed, which may admit waiting sessions.
 * The caller drives the loop with cvc_server_poll (no hidden threads).
 * Buffers in a request are the caller's and must stay valid until its
 * completion is returned.                                                   */
typedef struct cvc_server cvc_server;

typedef struct {
    size_t budget_bytes;   /* device bytes the server may hold (shards' state and workspace) */
    int slots_per_shard;   /* 1..256 */
    int steps_in_flight;   /* steps a shard may have queued on the device at once, 1..8 (0: 1).
                              With 2 or more, requests that arrive while a step runs are queued
                              behind it at once instead of after its completion is collected;
                              a step skips the work of the slots that have no request in it.
                              Shards of frames up to 352x288 run on the highest-priority
                              stream, up to 640x480 on a middle one, larger on the lowest.  */
} cvc_server_config;

typedef struct {
    uint64_t tag;                /* the caller's tag of the request */
    int session;
    int kind;                    /* CVC_STEP_* of the request */
    cvc_status enc_status, dec_status;
    size_t out_len;
    int frame_type, dec_frame_type;
    int64_t t_submit_ns, t_launch_ns, t_done_ns;   /* cvc_server_now_ns clock */
} cvc_server_completion;

typedef struct {
    size_t budget_bytes, used_bytes, peak_used_bytes;
    int shards, active_sessions, waiting_sessions;
    long long steps, requests_done, requests_queued;
} cvc_server_stats;

/* host steady clock (CLOCK_MONOTONIC) in nanoseconds */
int64_t cvc_server_now_ns(void);
cvc_status cvc_server_create(const cvc_server_config* config, cvc_server** out);
/* waits for in-flight steps, frees everything */
cvc_status cvc_server_destroy(cvc_server* server);
/* open a session; NOMEM if one shard of its parameters exceeds the whole budget */
cvc_status cvc_server_open(cvc_server* server, const cvc_params* params, int* session);
/* no further submits; the slot is freed after the session's last completion */
cvc_status cvc_server_close(cvc_server* server, int session);
/* queue one request (io as for cvc_batch_step; `kind` CVC_STEP_*).
 * INVALID_ARG (nothing queued) for a closed session or buffers that do not
 * fit the session's frame size.                                             */
cvc_status cvc_server_submit(cvc_server* server, int session, int kind, const cvc_batch_io* io, uint64_t tag);
/* Run the loop once: collect finished steps, free and admit, launch steps
 * for idle shards with queued requests; then, if no completion is ready,
 * wait up to wait_us microseconds for one.  Copies up to max_out
 * completions to out (*n_out of them); the rest stay for the next poll.    */
cvc_status cvc_server_poll(cvc_server* server, int wait_us, cvc_server_completion* out, int max_out, int* n_out);
cvc_status cvc_server_get_stats(const cvc_server* server, cvc_server_stats* out);

/* --------------------------------------------------------------- tracing
 * Per-stage GPU time of a codec (the per-operation breakdown of §4.2),
 * measured with CUDA events recorded on the call's stream around each stage
 * and read back at the synchronisation that encode / decode already do.
 * Stages (index: name): 0 colour+chroma+pad, 1 LP analysis, 2 DFB analysis,
 * 3 quantise+K/P, 4 RLE+bitstream, 5 bitstream parse+un-RLE,
 * 6 inverse K/P+dequantise, 7 DFB synthesis, 8 LP synthesis, 9 chroma
 * upsampling+colour.                                                       */
#define CVC_NUM_STAGES 10

/* enable (on != 0) or disable stage timing; enabling clears the totals */
cvc_status cvc_codec_set_timing(cvc_codec* codec, int on);
/* accumulated milliseconds and kernel launches per stage since enabling;
 * ms and launches each hold CVC_NUM_STAGES entries (either may be NULL)     */
cvc_status cvc_codec_timing(const cvc_codec* codec, double* ms, long long* launches);

/* Kernels this library has launched in this process (all contexts). */
unsigned long long cvc_kernel_launches(void);

/* ------------------------------------------------ allocation-free pyramid
 * The paper has no counterpart: this is a deployment variant for callers
 * that cannot allocate device memory while they run (a fixed memory budget
 * handed out up front, or a context where the CUDA allocator is off limits)
 * and therefore cannot create a cvc_ct_plan.
 *
 * Computes exactly what cvc_ct_forward computes for a plan with
 * dirs_log2 = {0, ..., 0}: the Laplacian pyramid of one dense h x w float
 * plane d_x, written to d_coeffs in that plan's layout (lowpass
 * (h>>L) x (w>>L), then the full-size detail of each level 1..L).  Both
 * buffers belong to the caller.  It calls no allocator: its scratch (the
 * intermediate lowpass images, one job record per level, the tile map) is a
 * 16 MiB file-scope __device__ array that every GPU loading the library holds
 * until the process exits.
 *   - Limits: h and w multiples of 2^levels; the intermediate lowpass
 *     images, sum_{j=1}^{L-1} (h>>j)(w>>j) floats (about h*w/3), must fit
 *     the array's 4,177,536-float workspace (planes up to ~12.5 Mpixel, e.g.
 *     4K UHD padded to 2176 x 3840), and the full-size plane may span at
 *     most 16,384 tiles of 64 x 64.  Larger planes return
 *     CVC_ERR_UNSUPPORTED before any device work.
 *   - The first call on each device looks up the array's device address
 *     (cudaGetSymbolAddress) with that device current and keeps it for the
 *     process; make that first call before any stream capture.  A
 *     cudaDeviceReset() of that device invalidates the kept address: do not
 *     call this entry point on a device after resetting it.
 *   - Each call writes its job records into the array with a one-block
 *     set-up kernel on `stream` (no host-to-device copy), then runs one
 *     launch per pyramid level.
 *   - Every call shares the one array: calls that overlap on the GPU (other
 *     streams, other host threads) race and corrupt each other.  Calls on a
 *     single stream are ordered and safe.
 * Asynchronous on `stream`.  Errors: INVALID_ARG, UNSUPPORTED, CUDA.        */
cvc_status cvc_lp_pyramid_forward_static(const float* d_x, int h, int w, int levels, float* d_coeffs,
                                         cvc_stream_t stream);

/* ------------------------------------------------------------ diagnostics
 * Host-only dump of the launch plan of a transform (no device call is
 * made, so it works without a GPU): the job tables of every launch of
 * `mode` & 255 (0 forward, 1 inverse, 2 adjoint of forward, 3 adjoint of
 * inverse) at fusion depth `mode` >> 8 (cvc_batch_set_fusion)
 * for a transform plan (params == NULL; h, w, levels, dirs_log2, batch as in
 * cvc_ct_plan_create) or for the planes of the codec streams params[0 ..
 * batch-1] (params != NULL: cvc_create for batch = 1, cvc_batch_create
 * otherwise; h, w, levels and dirs_log2 are ignored).  Layout written to buf, little
 * endian:
 *   u32 magic 0x43564350 ('CVCP'), u32 n_launches, u32 bytes of an LP-level
 *   job, u32 bytes of a DFB stage-1+2 job, u32 bytes of a DFB row-split job,
 *   u32 bytes of the trailing records (cvc_debug_scale_tables; else 0),
 *   u64 elems[4]   floats of the input, coefficient, workspace and output buffers,
 *   then per launch: u32 kind (0 = LP level, 1 = DFB stages 1-2, 2 = DFB stage
 *   >= 3), u32 njobs, and njobs job records (the library's job structures;
 *   DFB jobs carry their prototype length); or, for a pyramid-tail launch,
 *   u32 kind 3, u32 byte count, and the tail's tables: u32 planes, u32
 *   prototype length, then per plane i32 shared-memory floats, i32 stream,
 *   u32 steps, u32 0, and per step u32 kind (0, 1 or 2 as above), u32 1 for an LP
 *   step computed centred in single precision (the first level) else 0
 *   and the job record; the tail's own images are base 4.
 * Lets a test check, before any GPU run, that every access of every job
 * stays inside its buffer and that the tables compute the transform.
 * Returns CAPACITY with *used = bytes needed when cap is too small.          */
cvc_status cvc_debug_plan_tables(const cvc_params* params, int h, int w, int levels, const int* dirs_log2,
                                 int batch, int mode, void* buf, size_t cap, size_t* used);

/* The decoder back end at pyramid scale `scale` of the codec streams
 * params[0 .. n-1] (host only, no device call): the inverse transform's
 * launches over their sub-pyramids, in the format above with the header's
 * last u32 = bytes of one output record, followed by n output records
 *   {i32 H, W, Hc, Wc, rs_y, rs_c, src, blk0; i64 off[3]; f32 norm; i32 0}
 * (output frame and chroma size at the scale, plane row pitches, source
 * buffer 0 = reconstructed planes / 1 = decoded coefficients, first block,
 * Y/Co/Cg offsets, normalisation).  elems[] are those of the full decoder.
 * INVALID_ARG for a scale outside [0, max levels]; CAPACITY as above.       */
cvc_status cvc_debug_scale_tables(const cvc_params* params, int n, int scale, void* buf, size_t cap,
                                  size_t* used);

#ifdef __cplusplus
}
#endif
#endif
