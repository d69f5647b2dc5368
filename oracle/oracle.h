/*
 * oracle.h -- plain FP64 CPU oracle of the CVC contourlet codec hot path.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product library links, includes
 * or calls this code; only the test-suite, the smoke check and the CPU
 * baseline leg of the benchmark do.  It shares no code, header, table or
 * constant with the CUDA path.
 *
 * Every function follows one step of the method of Katsigiannis,
 * Papaioannou and Maroulis, "CVC: The Contourlet Video Compression
 * algorithm for real-time applications" (arXiv:1510.00561); the comment
 * above each definition names the section / equation / table it restates
 * and, where the paper is silent, the reading it takes.
 *
 * Floating point is double precision throughout, except where a float
 * value decides an integer (the quantiser, the final pixel rounding): that
 * decision is taken in single precision, the precision of the GPU path.
 */
#ifndef CVC_ORACLE_H
#define CVC_ORACLE_H
#include <stdint.h>

#define OR_MAX_LEVELS 6
#define OR_MAX_K 6
#define OR_MAX_SUB (1 + OR_MAX_LEVELS * 64)

/* status codes of the oracle (its own numbering) */
#define OR_OK 0
#define OR_EINVAL 1
#define OR_ECAPACITY 3
#define OR_EOVERFLOW 4
#define OR_ECORRUPT 5
#define OR_ESTATE 9
#define OR_MAX_RANGE 64

typedef struct {
    long off;   /* element offset inside the plane's coefficient block */
    int h, w;   /* subband rows, columns                               */
    int level;  /* 0 = lowpass, 1 = finest LP level ... L = coarsest    */
    int dir;    /* direction index in tree order (lowpass: 0)           */
    int kind;   /* 0 lowpass, 1 F_c wedge, 2 F_r wedge, 3 undivided detail (k=0), 4 quincunx half (k=1) */
} or_subband;

typedef struct {
    int H, W, L, k[OR_MAX_LEVELS];
    int nsub;                 /* lowpass + all directional subbands */
    or_subband sb[OR_MAX_SUB];
    long total;               /* coefficients of one plane */
} or_layout;

int or_modulus(int L, const int* k);
int or_layout_make(int H, int W, int L, const int* k, or_layout* out);

/* CDF 9/7 lowpass pair: h[0..8] = analysis taps at -4..4, g[0..6] = synthesis taps at -3..3 */
void or_cdf97(double* h, double* g);

/* Laplacian pyramid, one level (periodic extension), and adjoints */
void or_lp_analysis(const double* x, int H, int W, double* c, double* d);
void or_lp_synthesis(const double* c, const double* d, int H, int W, double* x);
void or_lp_analysis_adjoint(const double* cbar, const double* dbar, int H, int W, double* xbar);
void or_lp_synthesis_adjoint(const double* xbar, int H, int W, double* cbar, double* dbar);

/* directional filter bank with k stages on an H x W detail image.
 * mode 0: forward (analysis), 1: inverse, 2: adjoint of forward, 3: adjoint of inverse.
 * analysis direction (modes 0,3): plane -> subbands concatenated in tree order.
 * synthesis direction (modes 1,2): subbands -> plane.                              */
int or_dfb(int mode, const double* in, int H, int W, int k, double* out);
/* the same with an n-tap prototype, n = 4 (the one above), 6 or 8: the
 * Lagrange half-band interpolators (3, -25, 150, 150, -25, 3)/256 and
 * (-5, 49, -245, 1225, 1225, -245, 49, -5)/2048 at a = -5..5 / -7..7       */
int or_dfb_taps(int mode, const double* in, int H, int W, int k, int taps, double* out);

/* full contourlet transform on one plane, modes as above; coefficient layout of or_layout */
int or_ct(int mode, const double* in, int H, int W, int L, const int* k, double* out);
int or_ct_taps(int mode, const double* in, int H, int W, int L, const int* k, int taps, double* out);

/* colour, chroma and padding steps */
void or_ycocgr_forward(const uint8_t* rgb, long n, int16_t* y, int16_t* co, int16_t* cg);
void or_ycocgr_inverse(const int16_t* y, const int16_t* co, const int16_t* cg, long n, uint8_t* rgb);
void or_chroma_down(const int16_t* in, int H, int W, int16_t* out);
void or_chroma_up(const int16_t* in, int Hc, int Wc, int H, int W, int16_t* out);
void or_pad_mirror(const double* in, int H, int W, int Hp, int Wp, double* out);
/* Table 1 in its real-valued form with the paper's 8-bit storage (§3.1):
 * Y = (R + 2G + B)/4, Co = (R - B)/2, Cg = (2G - R - B)/4, each rounded half
 * away from zero; Co and Cg offset by +127 and clamped to [0, 255].  The
 * inverse removes the offset and applies R = Y + Co - Cg, G = Y + Cg,
 * B = Y - Co - Cg, clamped to [0, 255].                                    */
void or_ycocg8_forward(const uint8_t* rgb, long n, int16_t* y, int16_t* co, int16_t* cg);
void or_ycocg8_inverse(const int16_t* y, const int16_t* co, const int16_t* cg, long n, uint8_t* rgb);

/* quantiser of one value, single-precision decision (returns 0 on overflow flag set) */
int or_quantize(float c, int qp, float threshold, int is_lowpass, int levels, int* ovf);
/* the same under 8-bit storage (§3.6): the rounded quotient is clamped to
 * a byte, [-128, 127] for subbands and [0, 255] for the lowpass; single
 * precision                                                                */
int or_quantize8(float c, int qp, float threshold, int is_lowpass, int levels);

/* run-length coding of one row; returns tokens written */
long or_rle_row(const int16_t* row, int w, int16_t* tokens);
/* expand one component's tokens into n elements; returns OR_OK or OR_ECORRUPT */
int or_rle_expand(const int16_t* tokens, long ntok, int16_t* out, long n);

/* ------------------------------------------------- soft thresholding
 * Differentiable stand-in for the hard subband threshold of §3.5, used to
 * tune the thresholds by gradient descent: in directional subband s (layout
 * order, s = 0 .. nsub-2) y = sign(c) max(|c| - T[s], 0); the lowpass is
 * copied.  The vector-Jacobian product takes dL/dy and gives
 * dL/dc = dL/dy [|c| > T[s]] (lowpass: dL/dy) and
 * dL/dT[s] = -sum_{i in s} dL/dy_i sign(c_i) [|c_i| > T[s]], over `batch`
 * coefficient vectors of the layout.                                        */
void or_soft_threshold(const double* c, const or_layout* lay, int batch, const double* T, double* y);
void or_soft_threshold_vjp(const double* c, const or_layout* lay, int batch, const double* T, const double* g,
                           double* gc, double* gT);

/* ---------------------------------------------------------------- codec */
typedef struct or_codec or_codec;
or_codec* or_codec_create(int width, int height, int levels, const int* dirs, int qph, int qpl,
                          float threshold, int key_interval);
void or_codec_destroy(or_codec* c);
void or_codec_reset(or_codec* c);
long or_codec_coeff_count(const or_codec* c);      /* coefficients of the 3 planes */
long or_codec_max_stream(const or_codec* c);       /* worst-case stream bytes      */
int or_codec_ncomp(const or_codec* c);
/* padded plane sizes: out[0..3] = Hp, Wp, Hcp, Wcp */
void or_codec_dims(const or_codec* c, int* out);

/* colour + chroma + pad of one frame: float planes Y (Hp x Wp), Co, Cg (Hcp x Wcp) */
void or_codec_planes(const or_codec* c, const uint8_t* rgb, double* y, double* co, double* cg);

/* §3.2 motion estimation between the current and the previous frame's padded
 * luma planes (H x W, values 0..255): 16 x 16 blocks in raster order (the last
 * block row and column clipped to the plane); every displacement (dy, dx) in
 * [-range, range]^2 whose displaced block lies inside the plane is a
 * candidate; the smallest sum of squared differences wins (the MSE of the
 * block, whose size is the same for all its candidates); ties go to the
 * smaller |dy| + |dx|, then to the first candidate in raster order (dy, then
 * dx, ascending).  mv[2b] = dy, mv[2b + 1] = dx of block b.               */
void or_motion_search(const uint8_t* cur, const uint8_t* prev, int H, int W, int range, int8_t* mv);
/* P-frames with motion (§3.2, §3.7): range W in [0, OR_MAX_RANGE]; 0 keeps
 * zero-motion P-frames.  With W > 0 a P-frame (type byte 2) carries the
 * vectors of the luma blocks of its padded luma plane after its tokens (int8
 * dy, dx per block, raster order), and every component's residual is taken
 * against the motion-compensated prediction of the previous codes: element
 * (i, j) of a component whose element covers 2^ey x 2^ex luma samples uses
 * the vector of the block holding luma sample (i 2^ey, j 2^ex) (the last
 * block row / column for positions past the plane), scaled by 2^-ey, 2^-ex
 * with rounding half away from zero, and reads the previous code at the
 * displaced position clamped to the component.                              */
int or_codec_set_motion(or_codec* c, int range);
/* 8-bit storage (§3.1, §3.6), on != 0: the colour transform and quantiser
 * above, header byte 5 = 1; a decoder accepts only streams of its own
 * storage.  Default 0: YCoCg-R and int16 codes.                            */
int or_codec_set_storage8(or_codec* c, int on);
/* the DFB prototype length of the codec (4, the default, 6 or 8); header
 * byte 5 carries it in bits 1-2 (0, 1, 2), bit 0 being the 8-bit storage  */
int or_codec_set_taps(or_codec* c, int taps);

/* the entropy side of the encoder from given single-precision coefficients:
 * threshold, quantise, K/P differencing, state update, RLE, bitstream.      */
int or_encode_from_coeffs(or_codec* c, const float* coeffs, uint8_t* out, long cap,
                          long* out_len, int* frame_type);
/* the same with the frame's padded luma plane (Hp x Wp bytes), which motion
 * estimation needs (required when the codec has a motion range)            */
int or_encode_from_coeffs_luma(or_codec* c, const float* coeffs, const uint8_t* luma, uint8_t* out, long cap,
                               long* out_len, int* frame_type);
/* full encode: planes -> CT (FP64) -> single-precision decision -> entropy side.
 * coeffs_out (optional, FP64, or_codec_coeff_count values) receives the CT output. */
int or_encode(or_codec* c, const uint8_t* rgb, uint8_t* out, long cap, long* out_len,
              int* frame_type, double* coeffs_out);
/* full decode; planes_out (optional, FP64) receives the reconstructed padded planes */
int or_decode(or_codec* c, const uint8_t* in, long len, uint8_t* rgb, double* planes_out);
/* decode at scale s in [0, L] (§3.3): the decoder state advances for every
 * component as in or_decode, and the frame is reconstructed from the lowpass
 * and levels s+1..L only: the level-s approximation, normalised by 2^-s, as
 * ceil(H/2^s) x ceil(W/2^s) RGB.  planes_out receives the three normalised
 * (Hp>>s) x (Wp>>s), (Hcp>>s) x (Wcp>>s) planes. */
int or_decode_scaled(or_codec* c, const uint8_t* in, long len, int scale, uint8_t* rgb, double* planes_out);
/* a frame without its finest `drop` levels (§3.3: a receiver drops what refers
 * to resolutions above the one it wants): those components keep a zero token
 * count and lose their tokens, header bytes 26-27 hold `drop`.  Such a frame
 * decodes at scales >= drop only; after it the decoder state of levels
 * 1..drop is missing (a K-frame sets the missing levels to exactly its own
 * drop), and a P-frame decodes only at scales >= that floor.
 * Returns OR_OK, OR_EINVAL (drop < the frame's own drop or > L), OR_ECORRUPT,
 * OR_ECAPACITY (*out_len = bytes needed). */
int or_stream_drop(const or_codec* c, const uint8_t* in, long len, int drop, uint8_t* out, long cap,
                   long* out_len);

/* §3.9 DEFLATE: the cost (sum freq x length) of an optimal prefix code of n
 * symbols (Huffman's pairing); *depth = its longest code */
unsigned long long or_huffman_cost(const unsigned long* freq, int n, int* depth);
/* the frame inside a deflated frame (per-component raw DEFLATE streams after
 * the header, token counts, stream lengths and segment table, version byte
 * 2; or, CVC-NTS of §3.9, version byte 3, one stream of all the token bytes),
 * inflated with zlib; OR_ECORRUPT unless every stream inflates to exactly its
 * tokens */
int or_inflate_container(const or_codec* c, const uint8_t* in, long len, uint8_t* out, long cap, long* out_len);

#endif
