// codec_core.cuh -- the multi-stream codec core behind cvc_codec (one
// stream) and cvc_batch (many streams of any sizes).
//
// Every launch of an encode or decode step covers all streams of the core:
// the transform through one CtEngine over all their planes, the element-wise
// and row-wise stages through block maps.  Per-call arguments live in SCall
// records copied from pinned host memory at the start of the step, and the
// per-stream results come back through one copy at its end, so a step is a
// fixed launch sequence that is captured once in a CUDA graph and replayed
// for every frame.  The pinned records form a ring of CORE_RING slots, so
// that the host can fill the next calls while earlier ones are in flight.
//
// Coder state lives on the device (SCtl per stream) and stays consistent
// without host work between steps: a step writes the NEXT state buffers
// (est[1-ecur], dst[1-dcur]) and its last kernel flips ecur / dcur and
// advances the frame counters only for streams whose call succeeded, so a
// failed or skipped call leaves the stream exactly as it was, and calls can
// be queued back to back.
#pragma once
#include <memory>
#include <vector>

#include "k_codec.cuh"

namespace cvc {

enum StepMode { STEP_ENC = 1, STEP_DEC = 2, STEP_ENCDEC = 3 };

// launch shapes the autotuner may change (they change no result)
struct LaunchShape {
    int rle_rows;    // rows per block of the motion-compensation row kernels (one warp per row)
    int tok_blocks;  // blocks of the decoder's grid-stride token-tile kernels
};

// The decoder's back end at one pyramid scale s (§3.3: every LP scale can
// be decoded on its own).  Scale s keeps the lowpass and levels s+1..L of
// each plane, which are the coefficients of the (Hp >> s) x (Wp >> s)
// level-s lowpass image under an (L - s)-level transform; their inverse,
// normalised by 2^-s, is the output at ceil(H / 2^s) x ceil(W / 2^s).  A
// stream with L = s has no transform left: its lowpass bands are the planes.
// Scale 0 is the full decode (the core's own engine); every scale has its
// inverse colour table and its own step graphs.  Parsing, dequantisation
// and the decoder state cover every coefficient at every scale, so a stream
// may change scale from frame to frame.
struct ScalePlan {
    CtEngine eng;                    // s > 0: sub-pyramids of the streams with L > s
    std::vector<ScaleDesc> h_desc;   // one per stream (streams with L < s: unused)
    std::vector<int> h_blk;          // inverse colour launch: block -> stream
    ScaleDesc* d_desc = nullptr;     // in the core's arena
    int* d_blk = nullptr;
    cudaGraphExec_t gexec[4] = {nullptr, nullptr, nullptr, nullptr};   // index = StepMode
    long long gkernels[4] = {0, 0, 0, 0};
    ~ScalePlan();
};

struct Core {
    int n = 0;
    std::vector<cvc_params> prm;
    std::vector<SDesc> sd;
    std::vector<PlaneLayout> ly, lc;
    long long nplane = 0, ncoef = 0, sum_max_tok = 0, max_dtiles = 0;
    int nrows = 0, ncomp = 0, nplanes = 0, lowcols = 0, ntiles = 0;
    // host tables (kept for the size estimate and the upload)
    std::vector<PDesc> h_pd;
    std::vector<int> h_blk_colour, h_blk_plane, h_blk_motion;
    std::vector<long long> h_row_off, h_comp_elem;
    std::vector<int> h_row_w, h_row_stream, h_row_comp, h_comp_tile0, h_comp_stream;
    std::vector<long long> h_tile_off;         // RLE tiles (RleTiles)
    std::vector<int> h_tile_n, h_tile_w, h_tile_stream;
    std::vector<uint8_t> h_tile_low;
    std::vector<uint8_t> h_row_low, h_comp_low, h_comp_level, h_comp_plane, h_comp_ey, h_comp_ex;
    long long luma_total = 0, mv_pairs = 0;   // motion: luma bytes per buffer, vector pairs
    int motion_threads = 128;                  // block size of the motion search
    int motion_rmax = 0;                       // largest search range of the batch
    int motion_ws = 0, motion_smem = 0;        // its window row stride (a multiple of 4) and shared-memory bytes
    CtEngine eng;
    int max_levels = 0;
    std::vector<std::unique_ptr<ScalePlan>> scale;   // index = scale, 0 .. max_levels
    LaunchShape shape{8, 148 * 8};
    // device memory: one arena for everything but the engine's job tables
    void* arena = nullptr;
    size_t arena_bytes = 0;
    SDesc* d_sd = nullptr;
    SCall* d_sc = nullptr;
    SResult* d_rs = nullptr;
    PDesc* d_pd = nullptr;
    int *d_blk_colour = nullptr, *d_blk_plane = nullptr, *d_blk_motion = nullptr;
    long long *d_row_off = nullptr, *d_comp_elem = nullptr;
    int *d_row_w = nullptr, *d_row_stream = nullptr, *d_row_comp = nullptr, *d_comp_tile0 = nullptr,
        *d_comp_stream = nullptr;
    long long* d_tile_off = nullptr;
    int *d_tile_n = nullptr, *d_tile_w = nullptr, *d_tile_stream = nullptr;
    uint8_t* d_tile_low = nullptr;
    std::vector<int4> h_row_mc;
    int4* d_row_mc = nullptr;
    uint8_t *d_row_low = nullptr, *d_comp_low = nullptr, *d_comp_level = nullptr, *d_comp_plane = nullptr,
            *d_comp_ey = nullptr, *d_comp_ex = nullptr;
    uint8_t* d_luma[2] = {nullptr, nullptr};   // previous / current padded luma of streams with motion
    int8_t* d_mv = nullptr;                    // the encoder's motion vectors
    float *d_planes = nullptr, *d_rplanes = nullptr, *d_coef = nullptr, *d_dcoef = nullptr, *d_work = nullptr;
    int16_t *d_est_buf[2] = {nullptr, nullptr}, *d_dst_buf[2] = {nullptr, nullptr}, *d_res = nullptr;
    SCtl* d_ctl = nullptr;                     // device-resident coder state, one per stream
    uint32_t *d_tilecnt = nullptr, *d_tileoff = nullptr, *d_scan_tmp = nullptr;
    uint32_t *d_comp_tok = nullptr, *d_tok_base = nullptr, *d_scan_tmp2 = nullptr;
    // the decoder's token tiles: first tile per stream, codes per tile, their exclusive scan,
    // codes per component
    uint32_t *d_dtile_base = nullptr, *d_dtile_sum = nullptr, *d_dtile_pre = nullptr, *d_comp_codes = nullptr;
    // pinned per-call records: a ring of slots, each a call's SCall and SResult
    // arrays; ring_ev[k] completes when the last step that used slot k has
    // copied its results back.  h_sc / h_rs point at the current slot.
    static constexpr int CORE_RING = 8;
    SCall* ring_sc[CORE_RING] = {};
    SResult* ring_rs[CORE_RING] = {};
    cudaEvent_t ring_ev[CORE_RING] = {};
    bool ring_used[CORE_RING] = {};
    int ring_slot = 0;
    SCall* h_sc = nullptr;
    SResult* h_rs = nullptr;
    // streams whose coder state the next step resets (cvc_reset: stream-ordered)
    std::vector<uint8_t> pend_reset;
    // CUDA graphs of the step modes: one set per decoding scale (in ScalePlan)
    bool use_graphs = true;
    bool quant_pow2 = true;   // every stream's quantiser steps are powers of two
    cudaStream_t cap_stream = nullptr;
    // the pyramid tails run on a side stream, beside the DFB launches of the other levels
    // (fork / join events: [0] analysis, [1] synthesis)
    cudaStream_t side = nullptr;
    cudaEvent_t ev_fork[2] = {nullptr, nullptr}, ev_join[2] = {nullptr, nullptr};
    // stage timing (direct launches only)
    bool timing = false;
    cudaEvent_t ev[CVC_NUM_STAGES][2] = {};
    bool ev_used[CVC_NUM_STAGES] = {};
    double t_ms[CVC_NUM_STAGES] = {};
    long long t_launches[CVC_NUM_STAGES] = {};
    ~Core();
};

bool dirs_valid(int levels, const int* dirs);
bool codec_params_valid(const cvc_params* prm);
bool codec_geometry(const cvc_params* prm, ColourGeom* g);
std::vector<PlaneRef> codec_planes(const ColourGeom& g, int L, const int* dirs, int taps, long long plane_off,
                                   const long long poff[3], int stream);

// host tables and sizes, no device call; CVC_OK, INVALID_ARG or UNSUPPORTED
cvc_status core_plan(Core* c, const cvc_params* params, int n);
// device bytes core_alloc will allocate (after core_plan)
size_t core_device_bytes(const Core* c);
// allocate, upload, reset the state; CVC_OK or NOMEM / CUDA
cvc_status core_alloc(Core* c);
// reset the coder state of stream s (s < 0: all), from the next step on
void core_reset(Core* c, int s);
// start filling a new call: the next slot of the record ring (waits until the
// step that used it CORE_RING calls ago has returned its results), all
// streams' records cleared; false on a CUDA error
bool core_begin(Core* c);
// enqueue one step whose decoders output pyramid scale `scale` (the records
// in h_sc must be filled for that scale); no synchronisation
cvc_status core_enqueue(Core* c, int mode, cudaStream_t st, int scale = 0);
// capture the graph of a step mode ahead of its first use (no launch)
cvc_status core_capture(Core* c, int mode, int scale = 0);
// after the step completed: collect stage times
void core_collect(Core* c);
cvc_status core_set_timing(Core* c, bool on);
// drop the captured graphs (after a change of launch shape)
void core_drop_graphs(Core* c);
// the most coarse levels of each plane in its pyramid tail (0..CVC_MAX_LEVELS); rebuilds
// the transform tables of every scale and drops the graphs
cvc_status core_set_fusion(Core* c, int levels);
// threads per block of the row-split DFB launches: 0 (by launch size), 128 or 256
cvc_status core_set_dfb_threads(Core* c, int threads);

// fill the call record of stream s for a step (after core_begin); returns false on bad arguments
struct StreamIo {
    const uint8_t* rgb;
    size_t pitch;
    uint8_t* out;
    size_t out_cap;
    const uint8_t* in;
    size_t in_len;
    uint8_t* rgb_out;
    size_t pitch_out;
};
// (the decoder's output at pyramid scale `scale`, 0 <= scale <= the stream's levels)
bool core_fill_call(Core* c, int s, int mode, const StreamIo& io, int scale = 0);
// output size of stream s at a decoding scale
void core_scaled_size(const Core* c, int s, int scale, int* h, int* w);
// statuses of stream s after the step completed (the device has already
// advanced the coder state of the streams whose call succeeded)
void core_commit(Core* c, int s, int mode, cvc_status* enc, cvc_status* dec, size_t* out_len, int* type,
                 int* dec_type, unsigned* dec_index);
// the record-ring slot of the call being filled / last enqueued, and the
// statuses of stream s of the call that used slot `ring_slot` (for callers
// with several steps in flight)
int core_ring_slot(const Core* c);
void core_commit_at(Core* c, int ring_slot, int s, cvc_status* enc, cvc_status* dec, size_t* out_len, int* type,
                    int* dec_type, unsigned* dec_index);
// read and clear the first error of an asynchronous call of stream s (ordered on st; synchronises st)
cvc_status core_take_error(Core* c, int s, cudaStream_t st, cvc_status* err);

}  // namespace cvc
