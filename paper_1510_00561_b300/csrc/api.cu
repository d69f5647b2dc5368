// api.cu -- extern "C" entry points of libcvc.so (declared in include/cvc.h).
// The plain codec is a multi-stream core of one stream; a batch is a core of
// many.  Transform plans drive the contourlet engine directly.
#include <algorithm>
#include <atomic>
#include <cstring>
#include <new>
#include <vector>

#include "codec_core.cuh"
#include "k_deflate.cuh"
#include "k_soft.cuh"

using namespace cvc;

namespace cvc {
static std::atomic<unsigned long long> g_launches{0};
void note_launches(long long n) { g_launches.fetch_add((unsigned long long)n, std::memory_order_relaxed); }
}  // namespace cvc

namespace {

template <class T>
bool dalloc(std::vector<void*>& allocs, T** p, size_t n) {
    *p = nullptr;
    if (n == 0) n = 1;
    if (cudaMalloc((void**)p, n * sizeof(T)) != cudaSuccess) return false;
    allocs.push_back(*p);
    return true;
}

std::vector<PlaneRef> plan_planes(int h, int w, int levels, const int* dirs, int batch, long long total, int taps) {
    std::vector<PlaneRef> planes;
    for (int b = 0; b < batch; b++) {
        PlaneRef r;
        memset(&r, 0, sizeof(r));
        r.low_coef = -1;
        r.stream = -1;
        r.taps = taps;
        r.H = h;
        r.W = w;
        r.L = levels;
        for (int j = 0; j < levels; j++) r.k[j] = dirs[j];
        r.in.off = (long long)b * h * w;
        r.in.b = B_IN;
        r.in.rs = w;
        r.in.cs = 1;
        r.coef = (long long)b * total;
        planes.push_back(r);
    }
    return planes;
}

void fill_info(const Core& c, int s, cvc_codec_info_t* out) {
    const SDesc& D = c.sd[s];
    out->padded_height = D.cg.Hp;
    out->padded_width = D.cg.Wp;
    out->chroma_height = D.cg.Hc;
    out->chroma_width = D.cg.Wc;
    out->padded_chroma_height = D.cg.Hcp;
    out->padded_chroma_width = D.cg.Wcp;
    out->coeffs = D.ncoef;
    out->components = D.ncomp;
    out->max_stream_bytes = D.hdr_bytes + 2LL * D.max_tok + D.mv_bytes;
}

cvc_status make_core(Core* c, const cvc_params* params, int n) {
    cvc_status s = core_plan(c, params, n);
    if (s != CVC_OK) return s;
    return core_alloc(c);
}

// enqueue, wait, collect the stage times
cvc_status run_step(Core* c, int mode, cudaStream_t st, int scale = 0) {
    cvc_status s = core_enqueue(c, mode, st, scale);
    if (s != CVC_OK) return s;
    if (cudaStreamSynchronize(st) != cudaSuccess) {
        cudaGetLastError();
        return CVC_ERR_CUDA;
    }
    core_collect(c);
    return CVC_OK;
}

}  // namespace

// ====================================================================== plan
struct cvc_ct_plan {
    int h = 0, w = 0, L = 0, k[CVC_MAX_LEVELS] = {0}, batch = 0;
    PlaneLayout lay;
    CtEngine eng;
    float* d_work = nullptr;
    // soft thresholding: chunk jobs, first job of each directional subband, partial sums
    SoftJob* d_soft = nullptr;
    int* d_soft_first = nullptr;
    float* d_soft_partial = nullptr;
    int nsoft = 0, nsub = 0;
    std::vector<void*> allocs;
    ~cvc_ct_plan() {
        for (void* p : allocs) cudaFree(p);
    }
};

// ==================================================================== codecs
struct cvc_codec {
    Core core;
};
struct cvc_batch {
    Core core;
};

extern "C" {

const char* cvc_status_string(cvc_status s) {
    switch (s) {
        case CVC_OK: return "ok";
        case CVC_ERR_INVALID_ARG: return "invalid argument";
        case CVC_ERR_UNSUPPORTED: return "unsupported";
        case CVC_ERR_CAPACITY: return "output buffer too small";
        case CVC_ERR_OVERFLOW: return "quantised code outside int16";
        case CVC_ERR_CORRUPT: return "corrupt or mismatched bitstream";
        case CVC_ERR_CUDA: return "CUDA error";
        case CVC_ERR_TIMEOUT: return "device wait timed out";
        case CVC_ERR_NOMEM: return "out of memory";
        case CVC_ERR_STATE: return "P-frame without its reference frame";
    }
    return "unknown status";
}

int cvc_modulus(int levels, const int* dirs_log2) {
    if (!dirs_valid(levels, dirs_log2)) return 0;
    return modulus(levels, dirs_log2);
}

cvc_status cvc_ct_layout(int h, int w, int levels, const int* dirs_log2, cvc_ct_layout_t* out) {
    if (!out || !dirs_valid(levels, dirs_log2)) return CVC_ERR_INVALID_ARG;
    PlaneLayout L;
    if (!make_layout(h, w, levels, dirs_log2, &L)) return CVC_ERR_INVALID_ARG;
    memset(out, 0, sizeof(*out));
    out->height = h;
    out->width = w;
    out->levels = levels;
    for (int j = 0; j < levels; j++) out->dirs_log2[j] = dirs_log2[j];
    out->modulus = modulus(levels, dirs_log2);
    out->nsub = (int)L.sb.size();
    for (size_t i = 0; i < L.sb.size(); i++) {
        out->sub[i].off = L.sb[i].off;
        out->sub[i].h = L.sb[i].h;
        out->sub[i].w = L.sb[i].w;
        out->sub[i].level = L.sb[i].level;
        out->sub[i].dir = L.sb[i].dir;
        out->sub[i].kind = L.sb[i].kind;
    }
    out->total = L.total;
    return CVC_OK;
}

// ------------------------------------------------------------------ plan
cvc_status cvc_ct_plan_create(int h, int w, int levels, const int* dirs_log2, int batch, cvc_ct_plan** out) {
    return cvc_ct_plan_create_taps(h, w, levels, dirs_log2, batch, 4, out);
}

cvc_status cvc_ct_plan_create_taps(int h, int w, int levels, const int* dirs_log2, int batch, int dfb_taps,
                                   cvc_ct_plan** out) {
    if (!out) return CVC_ERR_INVALID_ARG;
    *out = nullptr;
    if (!dirs_valid(levels, dirs_log2) || batch < 1 ||
        (dfb_taps != 0 && dfb_taps != 4 && dfb_taps != 6 && dfb_taps != 8))
        return CVC_ERR_INVALID_ARG;
    cvc_ct_plan* p = new (std::nothrow) cvc_ct_plan();
    if (!p) return CVC_ERR_NOMEM;
    if (!make_layout(h, w, levels, dirs_log2, &p->lay)) {
        delete p;
        return CVC_ERR_INVALID_ARG;
    }
    p->h = h;
    p->w = w;
    p->L = levels;
    p->batch = batch;
    for (int j = 0; j < levels; j++) p->k[j] = dirs_log2[j];
    std::vector<PlaneRef> planes = plan_planes(h, w, levels, dirs_log2, batch, p->lay.total, dfb_taps);
    std::vector<SoftJob> sj;
    std::vector<int> sf;
    soft_jobs(p->lay, batch, &sj, &sf);
    p->nsoft = (int)sj.size();
    p->nsub = (int)sf.size() - 1;
    if (!engine_build(&p->eng, planes) || !dalloc(p->allocs, &p->d_work, (size_t)p->eng.work_elems) ||
        !dalloc(p->allocs, &p->d_soft, sj.size()) || !dalloc(p->allocs, &p->d_soft_first, sf.size()) ||
        !dalloc(p->allocs, &p->d_soft_partial, sj.size()) ||
        cudaMemcpy(p->d_soft, sj.data(), sj.size() * sizeof(SoftJob), cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemcpy(p->d_soft_first, sf.data(), sf.size() * sizeof(int), cudaMemcpyHostToDevice) != cudaSuccess ||
        lp_prepare() != cudaSuccess || dfb_prepare() != cudaSuccess || tail_prepare() != cudaSuccess) {
        cudaGetLastError();
        delete p;
        return CVC_ERR_NOMEM;
    }
    *out = p;
    return CVC_OK;
}

cvc_status cvc_ct_plan_destroy(cvc_ct_plan* plan) {
    delete plan;
    return CVC_OK;
}

cvc_status cvc_ct_plan_set_fusion(cvc_ct_plan* p, int levels) {
    if (!p || levels < 0 || levels > CVC_MAX_LEVELS) return CVC_ERR_INVALID_ARG;
    if (cudaDeviceSynchronize() != cudaSuccess) {
        cudaGetLastError();
        return CVC_ERR_CUDA;
    }
    p->eng.tail_levels = levels;
    const std::vector<PlaneRef> planes = p->eng.planes;
    if (!engine_build(&p->eng, planes, true)) {
        cudaGetLastError();
        return CVC_ERR_NOMEM;
    }
    return CVC_OK;
}

long long cvc_ct_plan_coeffs(const cvc_ct_plan* plan) { return plan ? plan->lay.total : 0; }

static cvc_status ct_run(cvc_ct_plan* p, Mode m, const float* in, float* out, cvc_stream_t stream) {
    if (!p || !in || !out) return CVC_ERR_INVALID_ARG;
    Bases B;
    memset(&B, 0, sizeof(B));
    B.p[B_WORK] = p->d_work;
    if (m == FWD || m == INV_ADJ) {
        B.p[B_IN] = const_cast<float*>(in);
        B.p[B_COEF] = out;
    } else {
        B.p[B_COEF] = const_cast<float*>(in);
        B.p[B_OUT] = out;
    }
    return engine_run(&p->eng, m, B, (cudaStream_t)stream) == cudaSuccess ? CVC_OK : CVC_ERR_CUDA;
}

cvc_status cvc_ct_forward(cvc_ct_plan* plan, const float* d_x, float* d_coeffs, cvc_stream_t stream) {
    return ct_run(plan, FWD, d_x, d_coeffs, stream);
}
cvc_status cvc_ct_inverse(cvc_ct_plan* plan, const float* d_coeffs, float* d_x, cvc_stream_t stream) {
    return ct_run(plan, INV, d_coeffs, d_x, stream);
}
cvc_status cvc_ct_forward_adjoint(cvc_ct_plan* plan, const float* d_coeffs_bar, float* d_x_bar, cvc_stream_t stream) {
    return ct_run(plan, FWD_ADJ, d_coeffs_bar, d_x_bar, stream);
}
cvc_status cvc_ct_inverse_adjoint(cvc_ct_plan* plan, const float* d_x_bar, float* d_coeffs_bar, cvc_stream_t stream) {
    return ct_run(plan, INV_ADJ, d_x_bar, d_coeffs_bar, stream);
}

int cvc_ct_plan_subbands(const cvc_ct_plan* plan) { return plan ? plan->nsub : 0; }

cvc_status cvc_ct_soft_threshold(cvc_ct_plan* p, const float* d_coeffs, const float* d_thresholds, float* d_out,
                                 cvc_stream_t stream) {
    if (!p || !d_coeffs || !d_thresholds || !d_out) return CVC_ERR_INVALID_ARG;
    if (launch_soft_fwd(p->d_soft, p->nsoft, d_coeffs, d_thresholds, d_out, (cudaStream_t)stream) != cudaSuccess) {
        cudaGetLastError();
        return CVC_ERR_CUDA;
    }
    note_launches(p->nsoft > 0);
    return CVC_OK;
}

cvc_status cvc_ct_soft_threshold_backward(cvc_ct_plan* p, const float* d_coeffs, const float* d_thresholds,
                                          const float* d_grad_out, float* d_grad_coeffs, float* d_grad_thresholds,
                                          cvc_stream_t stream) {
    if (!p || !d_coeffs || !d_thresholds || !d_grad_out || !d_grad_coeffs || !d_grad_thresholds)
        return CVC_ERR_INVALID_ARG;
    if (launch_soft_bwd(p->d_soft, p->nsoft, p->d_soft_first, p->nsub, d_coeffs, d_thresholds, d_grad_out,
                        d_grad_coeffs, d_grad_thresholds, p->d_soft_partial, (cudaStream_t)stream) != cudaSuccess) {
        cudaGetLastError();
        return CVC_ERR_CUDA;
    }
    note_launches((p->nsoft > 0) + (p->nsoft > 0 && p->nsub > 0));
    return CVC_OK;
}

// ----------------------------------------------------------------- codec
cvc_status cvc_create(const cvc_params* prm, cvc_codec** out) {
    if (!out) return CVC_ERR_INVALID_ARG;
    *out = nullptr;
    cvc_codec* c = new (std::nothrow) cvc_codec();
    if (!c) return CVC_ERR_NOMEM;
    cvc_status s = make_core(&c->core, prm, 1);
    if (s != CVC_OK) {
        delete c;
        return s;
    }
    *out = c;
    return CVC_OK;
}

cvc_status cvc_destroy(cvc_codec* c) {
    delete c;
    return CVC_OK;
}

cvc_status cvc_reset(cvc_codec* c) {
    if (!c) return CVC_ERR_INVALID_ARG;
    core_reset(&c->core, -1);
    return CVC_OK;
}

cvc_status cvc_codec_info(const cvc_codec* c, cvc_codec_info_t* out) {
    if (!c || !out) return CVC_ERR_INVALID_ARG;
    fill_info(c->core, 0, out);
    return CVC_OK;
}

cvc_status cvc_encode_frame(cvc_codec* c, const uint8_t* d_rgb, size_t pitch_bytes, uint8_t* d_out, size_t out_cap,
                            size_t* out_len, int* frame_type, cvc_stream_t stream) {
    if (!c || !d_rgb || !d_out || !out_len) return CVC_ERR_INVALID_ARG;
    StreamIo io{d_rgb, pitch_bytes, d_out, out_cap, nullptr, 0, nullptr, 0};
    if (!core_begin(&c->core)) return CVC_ERR_CUDA;
    if (!core_fill_call(&c->core, 0, STEP_ENC, io)) return CVC_ERR_INVALID_ARG;
    cvc_status s = run_step(&c->core, STEP_ENC, (cudaStream_t)stream);
    if (s != CVC_OK) return s;
    cvc_status es;
    int type = 0;
    core_commit(&c->core, 0, STEP_ENC, &es, nullptr, out_len, &type, nullptr, nullptr);
    if (frame_type) *frame_type = type;
    return es;
}

cvc_status cvc_decode_frame(cvc_codec* c, const uint8_t* d_in, size_t in_len, uint8_t* d_rgb, size_t pitch_bytes,
                            cvc_stream_t stream) {
    return cvc_decode_frame_scaled(c, d_in, in_len, 0, d_rgb, pitch_bytes, stream);
}

cvc_status cvc_decode_frame_scaled(cvc_codec* c, const uint8_t* d_in, size_t in_len, int scale, uint8_t* d_rgb,
                                   size_t pitch_bytes, cvc_stream_t stream) {
    if (!c || !d_in || !d_rgb) return CVC_ERR_INVALID_ARG;
    StreamIo io{nullptr, 0, nullptr, 0, d_in, in_len, d_rgb, pitch_bytes};
    if (!core_begin(&c->core)) return CVC_ERR_CUDA;
    if (!core_fill_call(&c->core, 0, STEP_DEC, io, scale)) return CVC_ERR_INVALID_ARG;
    cvc_status s = run_step(&c->core, STEP_DEC, (cudaStream_t)stream, scale);
    if (s != CVC_OK) return s;
    cvc_status ds;
    core_commit(&c->core, 0, STEP_DEC, nullptr, &ds, nullptr, nullptr, nullptr, nullptr);
    return ds;
}

// ---------------------------------------------------------- asynchronous calls
// The same steps without the host waiting: the outcome goes to device memory
// (written by the step's last kernel), and the coder state advances on the
// device, so calls queue back to back on a stream.

cvc_status cvc_encode_frame_async(cvc_codec* c, const uint8_t* d_rgb, size_t pitch_bytes, uint8_t* d_out,
                                  size_t out_cap, size_t* d_out_len, int* d_frame_type, cvc_status* d_status,
                                  cvc_stream_t stream) {
    if (!c || !d_rgb || !d_out) return CVC_ERR_INVALID_ARG;
    StreamIo io{d_rgb, pitch_bytes, d_out, out_cap, nullptr, 0, nullptr, 0};
    if (!core_begin(&c->core)) return CVC_ERR_CUDA;
    if (!core_fill_call(&c->core, 0, STEP_ENC, io)) return CVC_ERR_INVALID_ARG;
    SCall& C = c->core.h_sc[0];
    C.async = 1;
    C.out_len_dev = d_out_len;
    C.type_dev = d_frame_type;
    C.enc_status_dev = d_status;
    return core_enqueue(&c->core, STEP_ENC, (cudaStream_t)stream);
}

cvc_status cvc_decode_frame_async(cvc_codec* c, const uint8_t* d_in, size_t in_cap, const size_t* d_in_len, int scale,
                                  uint8_t* d_rgb, size_t pitch_bytes, cvc_status* d_status, cvc_stream_t stream) {
    if (!c || !d_in || !d_rgb) return CVC_ERR_INVALID_ARG;
    StreamIo io{nullptr, 0, nullptr, 0, d_in, in_cap, d_rgb, pitch_bytes};
    if (!core_begin(&c->core)) return CVC_ERR_CUDA;
    if (!core_fill_call(&c->core, 0, STEP_DEC, io, scale)) return CVC_ERR_INVALID_ARG;
    SCall& C = c->core.h_sc[0];
    C.async = 1;
    C.in_len_dev = d_in_len;
    C.dec_status_dev = d_status;
    return core_enqueue(&c->core, STEP_DEC, (cudaStream_t)stream, scale);
}

cvc_status cvc_get_error(cvc_codec* c, cvc_stream_t stream, cvc_status* status) {
    if (!c || !status) return CVC_ERR_INVALID_ARG;
    return core_take_error(&c->core, 0, (cudaStream_t)stream, status);
}

cvc_status cvc_stream_drop_levels(const cvc_params* params, const uint8_t* in, size_t in_len, int drop,
                                  uint8_t* out, size_t out_cap, size_t* out_len) {
    if (!params || !in || !out_len || !codec_params_valid(params)) return CVC_ERR_INVALID_ARG;
    ColourGeom g;
    PlaneLayout ly, lc;
    if (!codec_geometry(params, &g) || !make_layout(g.Hp, g.Wp, params->levels, params->dirs_log2, &ly) ||
        !make_layout(g.Hcp, g.Wcp, params->levels, params->dirs_log2, &lc))
        return CVC_ERR_UNSUPPORTED;
    // pyramid level of each component, in stream order (Y, Co, Cg; layout order)
    std::vector<int> level;
    for (int p = 0; p < 3; p++)
        for (const SubbandG& sb : (p == 0 ? ly : lc).sb) level.push_back(sb.kind == 0 ? 0 : sb.level);
    const size_t ncomp = level.size(), hdr = 32 + 4 * ncomp;
    auto rd32 = [&](size_t at) {
        return (uint32_t)in[at] | ((uint32_t)in[at + 1] << 8) | ((uint32_t)in[at + 2] << 16) |
               ((uint32_t)in[at + 3] << 24);
    };
    if (in_len < hdr || memcmp(in, "CVC1", 4) != 0 || in[4] < 1 || in[4] > 3 || in[5] > 5 ||
        in[7] != params->levels || rd32(28) != ncomp)
        return CVC_ERR_CORRUPT;
    if (in[4] == 3) return CVC_ERR_UNSUPPORTED;   // CVC-NTS: one stream, no level can leave it
    const bool deflated = in[4] == 2;   // per-component DEFLATE streams (cvc_deflate_frame)
    const int d0 = in[26] | (in[27] << 8);
    if (drop < d0 || drop > params->levels) return CVC_ERR_INVALID_ARG;
    if (deflated && in_len < hdr + 4 * ncomp) return CVC_ERR_CORRUPT;
    // pass 1 (reads only): the sizes of what stays
    unsigned long long all = 0, keep = 0, nseg = 0, kseg = 0, sbytes = 0, kbytes = 0;
    for (size_t j = 0; j < ncomp; j++) {
        const uint32_t n = rd32(32 + 4 * j);
        const bool kept = level[j] == 0 || level[j] > drop;
        const unsigned long long segs = (2ULL * n + 255) / 256;
        all += n;
        nseg += segs;
        if (kept) {
            keep += n;
            kseg += segs;
        }
        if (deflated) {
            const uint32_t nb = rd32(hdr + 4 * j);
            sbytes += nb;
            if (kept) kbytes += nb;
        }
    }
    // a P-frame with motion carries its vectors after the tokens (or streams); they stay
    unsigned long long mvb = 0;
    if (in[6] == 2) {
        if (params->motion_range == 0) return CVC_ERR_CORRUPT;
        mvb = 2ULL * ((g.Hp + 15) / 16) * ((g.Wp + 15) / 16);
    }
    auto pad4 = [](unsigned long long v) { return (v + 3) & ~3ULL; };
    const unsigned long long body_in = deflated ? 4ULL * ncomp + pad4(2 * nseg) + sbytes : 2 * all;
    const unsigned long long body_out = deflated ? 4ULL * ncomp + pad4(2 * kseg) + kbytes : 2 * keep;
    if (hdr + body_in + mvb > in_len) return CVC_ERR_CORRUPT;
    *out_len = hdr + body_out + mvb;
    if (!out || out_cap < *out_len) return CVC_ERR_CAPACITY;
    // pass 2: every section moves forward (or stays), so `out` may be `in`
    memmove(out, in, 32);
    out[26] = (uint8_t)(drop & 255);
    out[27] = (uint8_t)(drop >> 8);
    if (!deflated) {
        size_t src = hdr, dst = hdr;
        for (size_t j = 0; j < ncomp; j++) {
            const uint32_t n = rd32(32 + 4 * j);
            const bool kept = level[j] == 0 || level[j] > drop;
            const uint32_t w = kept ? n : 0;
            memcpy(out + 32 + 4 * j, &w, 4);   // little-endian host
            if (kept) {
                memmove(out + dst, in + src, 2 * (size_t)n);
                dst += 2 * (size_t)n;
            }
            src += 2 * (size_t)n;
        }
        memmove(out + dst, in + src, (size_t)mvb);
        return CVC_OK;
    }
    // deflated frame: counts and stream lengths of dropped components become 0, their
    // segment entries and streams go
    std::vector<uint32_t> cnt(ncomp), nbs(ncomp);
    for (size_t j = 0; j < ncomp; j++) {
        cnt[j] = rd32(32 + 4 * j);
        nbs[j] = rd32(hdr + 4 * j);
    }
    const size_t seg_in = hdr + 4 * ncomp, str_in = seg_in + (size_t)pad4(2 * nseg);
    const size_t seg_out = seg_in, str_out = seg_out + (size_t)pad4(2 * kseg);
    size_t si = seg_in, so = seg_out;
    for (size_t j = 0; j < ncomp; j++) {
        const bool kept = level[j] == 0 || level[j] > drop;
        const uint32_t w = kept ? cnt[j] : 0, b = kept ? nbs[j] : 0;
        memcpy(out + 32 + 4 * j, &w, 4);
        memcpy(out + hdr + 4 * j, &b, 4);
        const size_t segb = 2 * (size_t)((2ULL * cnt[j] + 255) / 256);
        if (kept) {
            memmove(out + so, in + si, segb);
            so += segb;
        }
        si += segb;
    }
    for (; so < str_out; so++) out[so] = 0;
    size_t src = str_in, dst = str_out;
    for (size_t j = 0; j < ncomp; j++) {
        const bool kept = level[j] == 0 || level[j] > drop;
        if (kept) {
            memmove(out + dst, in + src, nbs[j]);
            dst += nbs[j];
        }
        src += nbs[j];
    }
    memmove(out + dst, in + src, (size_t)mvb);
    return CVC_OK;
}

cvc_status cvc_codec_set_timing(cvc_codec* c, int on) {
    if (!c) return CVC_ERR_INVALID_ARG;
    return core_set_timing(&c->core, on != 0);
}

cvc_status cvc_codec_timing(const cvc_codec* c, double* ms, long long* launches) {
    if (!c) return CVC_ERR_INVALID_ARG;
    for (int s = 0; s < CVC_NUM_STAGES; s++) {
        if (ms) ms[s] = c->core.t_ms[s];
        if (launches) launches[s] = c->core.t_launches[s];
    }
    return CVC_OK;
}

unsigned long long cvc_kernel_launches(void) { return g_launches.load(); }

cvc_status cvc_codec_inspect(const cvc_codec* c, int which, float* d_out, size_t cap_elems, cvc_stream_t stream) {
    if (!c || !d_out || which < 0 || which > 2) return CVC_ERR_INVALID_ARG;
    const Core& k = c->core;
    const float* src = which == 0 ? k.d_planes : (which == 1 ? k.d_coef : k.d_rplanes);
    size_t n = (size_t)(which == 1 ? k.ncoef : k.nplane);
    if (cap_elems < n) return CVC_ERR_INVALID_ARG;
    return cudaMemcpyAsync(d_out, src, n * 4, cudaMemcpyDeviceToDevice, (cudaStream_t)stream) == cudaSuccess
               ? CVC_OK
               : CVC_ERR_CUDA;
}

// --------------------------------------------------------------- DEFLATE
struct cvc_deflate_ctx {
    int ncomp = 0, max_seg = 0, max_grp = 0, max_frames = 0;
    int nts = 0;                        // deflate into one stream per frame (CVC-NTS)
    long long hdr_bytes = 0, mv_bytes = 0;
    void* arena = nullptr;
    DflScratch* d_S = nullptr;          // max_frames scratch records
    std::vector<DflScratch> ptrs;       // host copies of their device pointers
    DflFrame* d_fr = nullptr;           // the frames of a call
    DflFrame* h_fr = nullptr;           // pinned staging of d_fr
    DflScratch* h_S = nullptr;          // pinned: the scalars come back through it
    uint32_t *segbits = nullptr, *segoff = nullptr, *scan_tmp = nullptr;   // all frames
    ~cvc_deflate_ctx() {
        if (arena) cudaFree(arena);
        if (h_S) cudaFreeHost(h_S);
        if (h_fr) cudaFreeHost(h_fr);
    }
};

cvc_status cvc_deflate_create_batch(const cvc_params* params, int max_frames, cvc_deflate_ctx** out) {
    if (!out || max_frames < 1 || max_frames > 4096) return CVC_ERR_INVALID_ARG;
    *out = nullptr;
    Core core;   // the stream's layout: component count, token bound (host only)
    cvc_status s = core_plan(&core, params, 1);
    if (s != CVC_OK) return s;
    const SDesc& D = core.sd[0];
    cvc_deflate_ctx* x = new (std::nothrow) cvc_deflate_ctx();
    if (!x) return CVC_ERR_NOMEM;
    x->ncomp = D.ncomp;
    x->hdr_bytes = D.hdr_bytes;
    x->mv_bytes = D.mv_bytes;
    x->max_frames = max_frames;
    const long long segs = (2 * D.max_tok + DFL_SEG - 1) / DFL_SEG + D.ncomp;
    if (segs * max_frames > (1LL << 30)) {
        delete x;
        return CVC_ERR_UNSUPPORTED;
    }
    x->max_seg = (int)segs;
    x->max_grp = (int)((segs + DFL_GRP - 1) / DFL_GRP) + D.ncomp;
    const size_t n = (size_t)x->ncomp, m = (size_t)x->max_seg, F = (size_t)max_frames;
    size_t off = 0;
    auto take = [&](size_t bytes) {
        off = (off + 255) & ~size_t(255);
        const size_t at = off;
        off += std::max<size_t>(bytes, 1);
        return at;
    };
    const size_t o_S = take(F * sizeof(DflScratch)), o_fr = take(F * sizeof(DflFrame)),
                 o_sb = take((F * (m + 1)) * 4), o_so = take((F * (m + 1) + 1) * 4),
                 o_tmp = take(((F * (m + 1) + 2047) / 2048 + 8) * 4);
    std::vector<size_t> o_comp(F), o_hist(F), o_len(F), o_code(F), o_hdr(F), o_dc(F), o_ds(F), o_dt(F);
    for (size_t f = 0; f < F; f++) {
        o_comp[f] = take((n + 1) * sizeof(DflComp));
        o_hist[f] = take(n * DFL_NLIT * 4);
        o_len[f] = take(n * DFL_NLIT);
        o_code[f] = take(n * DFL_NLIT * 2);
        o_hdr[f] = take(n * DFL_HDR_BYTES);
        o_dc[f] = take(n * 16 * 2);
        o_ds[f] = take(n * DFL_NSYM * 2);
        o_dt[f] = take(n * (1 << DFL_LUT) * 2);
    }
    if (cudaMalloc(&x->arena, off) != cudaSuccess ||
        cudaMallocHost((void**)&x->h_S, F * sizeof(DflScratch)) != cudaSuccess ||
        cudaMallocHost((void**)&x->h_fr, F * sizeof(DflFrame)) != cudaSuccess) {
        cudaGetLastError();
        delete x;
        return CVC_ERR_NOMEM;
    }
    char* b = static_cast<char*>(x->arena);
    x->d_S = reinterpret_cast<DflScratch*>(b + o_S);
    x->d_fr = reinterpret_cast<DflFrame*>(b + o_fr);
    x->segbits = reinterpret_cast<uint32_t*>(b + o_sb);
    x->segoff = reinterpret_cast<uint32_t*>(b + o_so);
    x->scan_tmp = reinterpret_cast<uint32_t*>(b + o_tmp);
    x->ptrs.assign(F, DflScratch{});
    for (size_t f = 0; f < F; f++) {
        DflScratch& S = x->ptrs[f];
        memset(&S, 0, sizeof(S));
        S.comp = reinterpret_cast<DflComp*>(b + o_comp[f]);
        S.hist = reinterpret_cast<uint32_t*>(b + o_hist[f]);
        S.len = reinterpret_cast<uint8_t*>(b + o_len[f]);
        S.code = reinterpret_cast<uint16_t*>(b + o_code[f]);
        S.hdr = reinterpret_cast<uint8_t*>(b + o_hdr[f]);
        S.dcount = reinterpret_cast<uint16_t*>(b + o_dc[f]);
        S.dsym = reinterpret_cast<uint16_t*>(b + o_ds[f]);
        S.dtab = reinterpret_cast<uint16_t*>(b + o_dt[f]);
        S.segbits = x->segbits + f * (m + 1);
        S.segoff = x->segoff + f * (m + 1);
    }
    if (cudaMemcpy(x->d_S, x->ptrs.data(), F * sizeof(DflScratch), cudaMemcpyHostToDevice) != cudaSuccess) {
        cudaGetLastError();
        delete x;
        return CVC_ERR_CUDA;
    }
    *out = x;
    return CVC_OK;
}

cvc_status cvc_deflate_create(const cvc_params* params, cvc_deflate_ctx** out) {
    return cvc_deflate_create_batch(params, 1, out);
}

cvc_status cvc_deflate_set_nts(cvc_deflate_ctx* ctx, int on) {
    if (!ctx) return CVC_ERR_INVALID_ARG;
    ctx->nts = on != 0;
    return CVC_OK;
}

cvc_status cvc_deflate_destroy(cvc_deflate_ctx* ctx) {
    delete ctx;
    return CVC_OK;
}

// per-frame statuses and lengths after a call; returns the first non-OK one
static cvc_status dfl_finish(cvc_deflate_ctx* x, int nf, cudaStream_t st, size_t* out_len, cvc_status* status,
                             long long launches) {
    if (cudaMemcpyAsync(x->h_S, x->d_S, nf * sizeof(DflScratch), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess) {
        cudaGetLastError();
        return CVC_ERR_CUDA;
    }
    note_launches(launches);
    cvc_status first = CVC_OK;
    for (int f = 0; f < nf; f++) {
        const DflScratch& S = x->h_S[f];
        cvc_status v = CVC_OK;
        if (S.err & DFL_INTERNAL) v = CVC_ERR_CUDA;
        else if (S.err & DFL_CORRUPT) v = CVC_ERR_CORRUPT;
        else if (S.err & DFL_CAPACITY) v = CVC_ERR_CAPACITY;
        out_len[f] = (size_t)S.total;
        if (status) status[f] = v;
        if (first == CVC_OK) first = v;
    }
    return first;
}

// stage the frame table of a call; false on bad arguments
static bool dfl_frames(cvc_deflate_ctx* x, int nf, const uint8_t* const* d_in, const size_t* in_len,
                       uint8_t* const* d_out, const size_t* out_cap, bool aligned_out, cudaStream_t st) {
    if (!x || nf < 1 || nf > x->max_frames || !d_in || !in_len || !d_out || !out_cap) return false;
    for (int f = 0; f < nf; f++) {
        if (!d_in[f] || !d_out[f] || (aligned_out && ((uintptr_t)d_out[f] & 3))) return false;
        // whole words only: the streams are OR-ed in 32-bit words
        x->h_fr[f] = DflFrame{d_in[f], (long long)std::min<size_t>(in_len[f], (size_t)1 << 62), d_out[f],
                              (long long)(std::min<size_t>(out_cap[f], (size_t)1 << 62) & ~(size_t)3), x->d_S + f};
    }
    return cudaMemcpyAsync(x->d_fr, x->h_fr, nf * sizeof(DflFrame), cudaMemcpyHostToDevice, st) == cudaSuccess;
}

cvc_status cvc_deflate_frames(cvc_deflate_ctx* x, int nf, const uint8_t* const* d_in, const size_t* in_len,
                              uint8_t* const* d_out, const size_t* out_cap, size_t* out_len, cvc_status* status,
                              cvc_stream_t stream) {
    cudaStream_t st = (cudaStream_t)stream;
    if (!out_len || !dfl_frames(x, nf, d_in, in_len, d_out, out_cap, true, st)) return CVC_ERR_INVALID_ARG;
    const DflArgs a{x->d_fr, x->hdr_bytes, x->mv_bytes, x->ncomp, x->max_seg, x->max_grp, x->nts};
    const dim3 one(1, nf), strs(x->nts ? 1 : x->ncomp, nf), grps(x->max_grp, nf);
    k_dfl_plan<<<one, 256, 0, st>>>(a);
    k_dfl_hist<<<grps, 256, 0, st>>>(a);
    k_dfl_code<<<strs, 256, 0, st>>>(a);
    k_dfl_layout<<<one, 256, 0, st>>>(a);
    k_dfl_seglen<<<grps, 256, 0, st>>>(a);
    // one scan over every frame's slice; each frame only takes differences inside it
    if (exclusive_scan(x->segbits, (uint32_t)(nf * (x->max_seg + 1)), x->segoff, x->scan_tmp, st) != cudaSuccess) {
        cudaGetLastError();
        return CVC_ERR_CUDA;
    }
    k_dfl_zero<<<dim3(64, nf), 256, 0, st>>>(a);
    k_dfl_write<<<grps, 256, 0, st>>>(a);
    k_dfl_tables<<<dim3(16, nf), 256, 0, st>>>(a);
    if (cudaGetLastError() != cudaSuccess) return CVC_ERR_CUDA;
    return dfl_finish(x, nf, st, out_len, status, 11);
}

cvc_status cvc_inflate_frames(cvc_deflate_ctx* x, int nf, const uint8_t* const* d_in, const size_t* in_len,
                              uint8_t* const* d_out, const size_t* out_cap, size_t* out_len, cvc_status* status,
                              cvc_stream_t stream) {
    cudaStream_t st = (cudaStream_t)stream;
    if (!out_len || !dfl_frames(x, nf, d_in, in_len, d_out, out_cap, false, st)) return CVC_ERR_INVALID_ARG;
    const DflArgs a{x->d_fr, x->hdr_bytes, x->mv_bytes, x->ncomp, x->max_seg, x->max_grp, 0};
    const dim3 one(1, nf), comps(x->ncomp, nf), grps(x->max_grp, nf);
    k_ifl_plan<<<one, 256, 0, st>>>(a);
    k_ifl_seglen<<<dim3((x->max_seg + 255) / 256, nf), 256, 0, st>>>(a);
    if (exclusive_scan(x->segbits, (uint32_t)(nf * (x->max_seg + 1)), x->segoff, x->scan_tmp, st) != cudaSuccess) {
        cudaGetLastError();
        return CVC_ERR_CUDA;
    }
    k_ifl_tables<<<comps, 128, 0, st>>>(a);
    k_ifl_decode<<<grps, 256, 0, st>>>(a);
    k_ifl_finish<<<dim3(16, nf), 256, 0, st>>>(a);
    if (cudaGetLastError() != cudaSuccess) return CVC_ERR_CUDA;
    return dfl_finish(x, nf, st, out_len, status, 8);
}

cvc_status cvc_deflate_frame(cvc_deflate_ctx* x, const uint8_t* d_in, size_t in_len, uint8_t* d_out, size_t out_cap,
                             size_t* out_len, cvc_stream_t stream) {
    if (!x || !d_in || !d_out || !out_len) return CVC_ERR_INVALID_ARG;
    return cvc_deflate_frames(x, 1, &d_in, &in_len, &d_out, &out_cap, out_len, nullptr, stream);
}

cvc_status cvc_inflate_frame(cvc_deflate_ctx* x, const uint8_t* d_in, size_t in_len, uint8_t* d_out, size_t out_cap,
                             size_t* out_len, cvc_stream_t stream) {
    if (!x || !d_in || !d_out || !out_len) return CVC_ERR_INVALID_ARG;
    return cvc_inflate_frames(x, 1, &d_in, &in_len, &d_out, &out_cap, out_len, nullptr, stream);
}

// --------------------------------------------------------------- batches
cvc_status cvc_batch_create(const cvc_params* params, int n, cvc_batch** out) {
    if (!out) return CVC_ERR_INVALID_ARG;
    *out = nullptr;
    if (!params || n < 1) return CVC_ERR_INVALID_ARG;
    cvc_batch* b = new (std::nothrow) cvc_batch();
    if (!b) return CVC_ERR_NOMEM;
    cvc_status s = make_core(&b->core, params, n);
    if (s != CVC_OK) {
        delete b;
        return s;
    }
    *out = b;
    return CVC_OK;
}

cvc_status cvc_batch_destroy(cvc_batch* b) {
    delete b;
    return CVC_OK;
}

cvc_status cvc_batch_device_bytes(const cvc_params* params, int n, size_t* bytes) {
    if (!bytes || !params || n < 1) return CVC_ERR_INVALID_ARG;
    Core c;
    cvc_status s = core_plan(&c, params, n);
    if (s != CVC_OK) return s;
    *bytes = core_device_bytes(&c);
    return CVC_OK;
}

cvc_status cvc_batch_info(const cvc_batch* b, int i, cvc_codec_info_t* out) {
    if (!b || !out || i < 0 || i >= b->core.n) return CVC_ERR_INVALID_ARG;
    fill_info(b->core, i, out);
    return CVC_OK;
}

cvc_status cvc_batch_reset(cvc_batch* b, int i) {
    if (!b || i >= b->core.n) return CVC_ERR_INVALID_ARG;
    core_reset(&b->core, i < 0 ? -1 : i);
    return CVC_OK;
}

static bool batch_fill(Core* c, int what, const cvc_batch_io* io, int scale = 0) {
    for (int s = 0; s < c->n; s++) {
        const cvc_batch_io& x = io[s];
        StreamIo sio{x.d_rgb, x.pitch_bytes, x.d_out, x.out_cap, x.d_in, x.in_len, x.d_rgb_out, x.pitch_out};
        if (!core_fill_call(c, s, what, sio, scale)) return false;
    }
    return true;
}

cvc_status cvc_batch_step(cvc_batch* b, int what, const cvc_batch_io* io, cvc_batch_result* res,
                          cvc_stream_t stream) {
    return cvc_batch_step_scaled(b, what, io, 0, res, stream);
}

cvc_status cvc_batch_step_scaled(cvc_batch* b, int what, const cvc_batch_io* io, int scale, cvc_batch_result* res,
                                 cvc_stream_t stream) {
    if (!b || !io || !res || what < CVC_STEP_ENCODE || what > CVC_STEP_ENCODE_DECODE) return CVC_ERR_INVALID_ARG;
    Core* c = &b->core;
    if (!core_begin(c)) return CVC_ERR_CUDA;
    if (!batch_fill(c, what, io, scale)) return CVC_ERR_INVALID_ARG;
    cvc_status s = run_step(c, what, (cudaStream_t)stream, scale);
    if (s != CVC_OK) return s;
    cvc_status first = CVC_OK;
    for (int i = 0; i < c->n; i++) {
        cvc_batch_result& r = res[i];
        unsigned didx = 0;
        core_commit(c, i, what, &r.enc_status, &r.dec_status, &r.out_len, &r.frame_type, &r.dec_frame_type, &didx);
        r.dec_frame_index = didx;
        if (first == CVC_OK) first = r.enc_status != CVC_OK ? r.enc_status : r.dec_status;
    }
    return first;
}

cvc_status cvc_batch_step_async(cvc_batch* b, int what, const cvc_batch_io* io, const size_t* d_in_len, int scale,
                                cvc_batch_result* d_res, cvc_stream_t stream) {
    if (!b || !io || what < CVC_STEP_ENCODE || what > CVC_STEP_ENCODE_DECODE) return CVC_ERR_INVALID_ARG;
    Core* c = &b->core;
    if (!core_begin(c)) return CVC_ERR_CUDA;
    if (!batch_fill(c, what, io, scale)) return CVC_ERR_INVALID_ARG;
    for (int i = 0; i < c->n; i++) {
        SCall& C = c->h_sc[i];
        C.async = 1;
        C.in_len_dev = d_in_len ? d_in_len + i : nullptr;
        C.res_dev = d_res ? d_res + i : nullptr;
    }
    return core_enqueue(c, what, (cudaStream_t)stream, scale);
}

cvc_status cvc_batch_get_error(cvc_batch* b, int i, cvc_stream_t stream, cvc_status* status) {
    if (!b || !status || i < 0 || i >= b->core.n) return CVC_ERR_INVALID_ARG;
    return core_take_error(&b->core, i, (cudaStream_t)stream, status);
}

cvc_status cvc_batch_set_shape(cvc_batch* b, int rle_rows, int tok_blocks) {
    if (!b || rle_rows < 1 || rle_rows > 32 || tok_blocks < 1 || tok_blocks > 65535) return CVC_ERR_INVALID_ARG;
    b->core.shape = LaunchShape{rle_rows, tok_blocks};
    core_drop_graphs(&b->core);
    return CVC_OK;
}

cvc_status cvc_batch_set_graphs(cvc_batch* b, int on) {
    if (!b) return CVC_ERR_INVALID_ARG;
    b->core.use_graphs = on != 0;
    return CVC_OK;
}

cvc_status cvc_batch_set_timing(cvc_batch* b, int on) {
    if (!b) return CVC_ERR_INVALID_ARG;
    return core_set_timing(&b->core, on != 0);
}

cvc_status cvc_batch_timing(const cvc_batch* b, double* ms, long long* launches) {
    if (!b) return CVC_ERR_INVALID_ARG;
    for (int s = 0; s < CVC_NUM_STAGES; s++) {
        if (ms) ms[s] = b->core.t_ms[s];
        if (launches) launches[s] = b->core.t_launches[s];
    }
    return CVC_OK;
}

cvc_status cvc_batch_autotune(cvc_batch* b, int what, const cvc_batch_io* io, int reps, int* shape,
                              cvc_stream_t stream) {
    if (!b || !io || reps < 1 || what < CVC_STEP_ENCODE || what > CVC_STEP_ENCODE_DECODE) return CVC_ERR_INVALID_ARG;
    Core* c = &b->core;
    cudaStream_t st = (cudaStream_t)stream;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
        if (e0) cudaEventDestroy(e0);
        cudaGetLastError();
        return CVC_ERR_CUDA;
    }
    // time `reps` steps of one shape; no run commits its coder state, so
    // every run codes the same frame
    auto measure = [&](LaunchShape sh, float* ms) -> cvc_status {
        c->shape = sh;
        core_drop_graphs(c);
        if (!core_begin(c)) return CVC_ERR_CUDA;
        if (!batch_fill(c, what, io)) return CVC_ERR_INVALID_ARG;
        for (int i = 0; i < c->n; i++) c->h_sc[i].no_commit = 1;
        cvc_status s = core_enqueue(c, what, st);   // warm-up (and graph capture)
        if (s != CVC_OK) return s;
        cudaEventRecord(e0, st);
        for (int r = 0; r < reps && s == CVC_OK; r++) s = core_enqueue(c, what, st);
        cudaEventRecord(e1, st);
        if (s != CVC_OK) return s;
        if (cudaEventSynchronize(e1) != cudaSuccess || cudaEventElapsedTime(ms, e0, e1) != cudaSuccess) {
            cudaGetLastError();
            return CVC_ERR_CUDA;
        }
        return CVC_OK;
    };
    const int tok_cand[] = {148 * 2, 148 * 4, 148 * 8, 148 * 16, 148 * 32};
    const int rle_cand[] = {2, 4, 8, 16};
    LaunchShape best = c->shape;
    float best_ms = 0.f;
    cvc_status s = measure(best, &best_ms);
    // one coordinate at a time: token grid, then rows per block of the motion row kernels
    for (int t : tok_cand) {
        if (s != CVC_OK) break;
        LaunchShape sh{best.rle_rows, t};
        float ms = 0.f;
        s = measure(sh, &ms);
        if (s == CVC_OK && ms < best_ms) best = sh, best_ms = ms;
    }
    for (int r : rle_cand) {
        if (s != CVC_OK) break;
        LaunchShape sh{r, best.tok_blocks};
        float ms = 0.f;
        s = measure(sh, &ms);
        if (s == CVC_OK && ms < best_ms) best = sh, best_ms = ms;
    }
    // then the fusion depth: every level as its own launches, or tails of 1, 2 or as many
    // levels as fit
    const int fuse_cand[] = {0, 1, 2, CVC_MAX_LEVELS};
    int best_fuse = c->eng.tail_levels;
    for (int f : fuse_cand) {
        if (s != CVC_OK) break;
        if (f == best_fuse) continue;
        s = core_set_fusion(c, f);
        float ms = 0.f;
        if (s == CVC_OK) s = measure(best, &ms);
        if (s == CVC_OK && ms < best_ms) best_fuse = f, best_ms = ms;
    }
    if (s == CVC_OK && c->eng.tail_levels != best_fuse) s = core_set_fusion(c, best_fuse);
    // then the block width of the row-split DFB launches: by launch size, 128 or 256 threads
    const int dfbb_cand[] = {0, DFBB_THREADS, DFBB_THREADS_WIDE};
    int best_dfbb = c->eng.dfbb_threads;
    for (int t : dfbb_cand) {
        if (s != CVC_OK) break;
        if (t == best_dfbb) continue;
        s = core_set_dfb_threads(c, t);
        float ms = 0.f;
        if (s == CVC_OK) s = measure(best, &ms);
        if (s == CVC_OK && ms < best_ms) best_dfbb = t, best_ms = ms;
    }
    if (s == CVC_OK && c->eng.dfbb_threads != best_dfbb) s = core_set_dfb_threads(c, best_dfbb);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    c->shape = best;
    core_drop_graphs(c);
    if (shape) {
        shape[0] = best.rle_rows;
        shape[1] = best.tok_blocks;
        shape[2] = best_fuse;
        shape[3] = best_dfbb;
    }
    return s;
}

cvc_status cvc_batch_set_dfb_threads(cvc_batch* b, int threads) {
    if (!b) return CVC_ERR_INVALID_ARG;
    return core_set_dfb_threads(&b->core, threads);
}

cvc_status cvc_batch_set_fusion(cvc_batch* b, int levels) {
    if (!b) return CVC_ERR_INVALID_ARG;
    return core_set_fusion(&b->core, levels);
}

// the launches of one direction of an engine (and optional trailing
// records), in the cvc_debug_plan_tables format
static cvc_status dump_tables(const CtEngine& e, int mode, const unsigned long long elems_in[4], const void* tail,
                              size_t tail_n, size_t tail_sz, void* buf, size_t cap, size_t* used) {
    unsigned long long elems[4] = {elems_in[0], elems_in[1], elems_in[2], elems_in[3]};
    elems[2] = std::max(elems[2], (unsigned long long)e.work_elems);
    struct Item { int kind; const void* data; size_t n, sz; };
    std::vector<Item> items;
    const bool analysis = (mode == FWD || mode == INV_ADJ);
    auto push_lp = [&]() {
        for (auto& v : e.h_lp[mode]) items.push_back({0, v.data(), v.size(), sizeof(LpJob)});
    };
    auto push_dfb = [&]() {
        for (size_t i = 0; i < e.dfb[mode].size(); i++) {
            const LaunchDfb& L = e.dfb[mode][i];
            const size_t sz = L.kind == 0 ? sizeof(DfbAJob) : sizeof(DfbBJob);
            items.push_back({1 + L.kind, e.h_dfb[mode][i].data(), (size_t)L.njobs, sz});
        }
    };
    // pyramid-tail launches (kind 3): u32 nplanes, u32 ntaps; per plane i32 resident floats, i32 stream,
    // u32 nsteps, u32 0, then per step u32 kind (0 LP, 1 DFB stages 1-2, 2 DFB stage >= 3), u32 centred and
    // the job record; item size = blob bytes
    std::vector<std::vector<uint8_t>> blobs;
    for (const TailTables& T : e.h_tail[mode]) {
        std::vector<uint8_t> b;
        auto put = [&](const void* p, size_t n) {
            b.insert(b.end(), (const uint8_t*)p, (const uint8_t*)p + n);
        };
        uint32_t h2[2] = {(uint32_t)T.planes.size(), (uint32_t)T.ntaps};
        put(h2, 8);
        for (const TailPlane& P : T.planes) {
            int32_t ph[4] = {P.ws_floats, P.stream, P.nsteps, 0};
            put(ph, 16);
            for (int k = 0; k < P.nsteps; k++) {
                const TailStep& st = T.steps[(size_t)P.first_step + k];
                uint32_t sh[2] = {(uint32_t)st.kind, (uint32_t)st.centred};
                put(sh, 8);
                if (st.kind == 0) put(&T.lp[st.job], sizeof(LpJob));
                else if (st.kind == 1) put(&T.a[st.job], sizeof(DfbAJob));
                else put(&T.b[st.job], sizeof(DfbBJob));
            }
        }
        blobs.push_back(std::move(b));
    }
    auto push_tail = [&]() {
        for (auto& b : blobs) items.push_back({3, b.data(), b.size(), 1});
    };
    if (analysis) { push_lp(); push_tail(); push_dfb(); }
    else { push_dfb(); push_tail(); push_lp(); }
    size_t need = 24 + 32 + tail_n * tail_sz;
    for (const Item& it : items) need += 8 + it.n * it.sz;
    *used = need;
    if (!buf || cap < need) return CVC_ERR_CAPACITY;
    uint8_t* o = (uint8_t*)buf;
    uint32_t hdr[6] = {0x43564350u, (uint32_t)items.size(), (uint32_t)sizeof(LpJob), (uint32_t)sizeof(DfbAJob),
                       (uint32_t)sizeof(DfbBJob), (uint32_t)(tail_n ? tail_sz : 0)};
    memcpy(o, hdr, 24);
    memcpy(o + 24, elems, 32);
    size_t pos = 56;
    for (const Item& it : items) {
        uint32_t h2[2] = {(uint32_t)it.kind, (uint32_t)it.n};
        memcpy(o + pos, h2, 8);
        pos += 8;
        memcpy(o + pos, it.data, it.n * it.sz);
        pos += it.n * it.sz;
    }
    if (tail_n) memcpy(o + pos, tail, tail_n * tail_sz);
    return CVC_OK;
}

cvc_status cvc_debug_plan_tables(const cvc_params* params, int h, int w, int levels, const int* dirs_log2, int batch,
                                 int mode, void* buf, size_t cap, size_t* used) {
    const int fuse = mode >> 8;
    mode &= 255;
    if (!used || mode < 0 || mode > 3 || fuse > CVC_MAX_LEVELS) return CVC_ERR_INVALID_ARG;
    unsigned long long elems[4] = {0, 0, 0, 0};
    Core core;   // host tables only: core_plan makes no device call
    CtEngine plain;
    plain.tail_levels = fuse;
    const CtEngine* ep = nullptr;
    if (params) {
        cvc_status s = core_plan(&core, params, std::max(batch, 1));
        if (s != CVC_OK) return s;
        if (fuse) {
            core.eng.tail_levels = fuse;
            const std::vector<PlaneRef> planes = core.eng.planes;
            if (!engine_build(&core.eng, planes, false)) return CVC_ERR_UNSUPPORTED;
        }
        elems[0] = elems[3] = (unsigned long long)core.nplane;
        elems[1] = (unsigned long long)core.ncoef;
        ep = &core.eng;
    } else {
        PlaneLayout lay;
        if (!dirs_valid(levels, dirs_log2) || batch < 1 || !make_layout(h, w, levels, dirs_log2, &lay))
            return CVC_ERR_INVALID_ARG;
        std::vector<PlaneRef> planes = plan_planes(h, w, levels, dirs_log2, batch, lay.total, 4);
        if (!engine_build(&plain, planes, false)) return CVC_ERR_INVALID_ARG;
        elems[0] = elems[3] = (unsigned long long)batch * h * w;
        elems[1] = (unsigned long long)batch * lay.total;
        ep = &plain;
    }
    elems[2] = (unsigned long long)ep->work_elems;
    return dump_tables(*ep, mode, elems, nullptr, 0, 0, buf, cap, used);
}

cvc_status cvc_debug_scale_tables(const cvc_params* params, int n, int scale, void* buf, size_t cap,
                                  size_t* used) {
    if (!used || !params || n < 1) return CVC_ERR_INVALID_ARG;
    Core core;
    cvc_status s = core_plan(&core, params, n);
    if (s != CVC_OK) return s;
    if (scale < 0 || scale > core.max_levels) return CVC_ERR_INVALID_ARG;
    const ScalePlan& sp = *core.scale[scale];
    const unsigned long long elems[4] = {(unsigned long long)core.nplane, (unsigned long long)core.ncoef,
                                         (unsigned long long)core.eng.work_elems, (unsigned long long)core.nplane};
    return dump_tables(scale == 0 ? core.eng : sp.eng, INV, elems, sp.h_desc.data(), sp.h_desc.size(),
                       sizeof(ScaleDesc), buf, cap, used);
}

}  // extern "C"
