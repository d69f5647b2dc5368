// api.cu -- extern "C" entry points of libcvc.so (declared in include/cvc.h).
#include <algorithm>
#include <atomic>
#include <cstring>
#include <new>
#include <vector>

#include "k_codec.cuh"

using namespace cvc;

namespace cvc {
static std::atomic<unsigned long long> g_launches{0};
void note_launches(int n) { g_launches.fetch_add((unsigned long long)n, std::memory_order_relaxed); }
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

bool valid_dirs(int levels, const int* dirs) {
    if (levels < 1 || levels > CVC_MAX_LEVELS || !dirs) return false;
    for (int j = 0; j < levels; j++)
        if (dirs[j] < 0 || dirs[j] > CVC_MAX_DIRS_LOG2) return false;
    return true;
}

inline int round_up(int v, int m) { return (v + m - 1) / m * m; }

int grid_for(long long n, int block = 256) {
    long long g = (n + block - 1) / block;
    return (int)std::max(1LL, std::min(g, 148LL * 64));
}

// geometry shared by cvc_create and the plan dump
bool codec_geometry(const cvc_params* prm, ColourGeom* g) {
    const int M = modulus(prm->levels, prm->dirs_log2);
    g->H = prm->height;
    g->W = prm->width;
    g->Hp = round_up(g->H, M);
    g->Wp = round_up(g->W, M);
    g->Hc = (g->H + 1) / 2;
    g->Wc = (g->W + 1) / 2;
    g->Hcp = round_up(g->Hc, M);
    g->Wcp = round_up(g->Wc, M);
    // the mirror padding reaches back at most one plane size
    return !(g->Hp > 2 * g->H || g->Wp > 2 * g->W || g->Hcp > 2 * g->Hc || g->Wcp > 2 * g->Wc);
}

std::vector<PlaneRef> codec_planes(const ColourGeom& g, int L, const int* dirs, const FrameGeom& f) {
    std::vector<PlaneRef> planes(3);
    for (int p = 0; p < 3; p++) {
        memset(&planes[p], 0, sizeof(PlaneRef));
        planes[p].H = p == 0 ? g.Hp : g.Hcp;
        planes[p].W = p == 0 ? g.Wp : g.Wcp;
        planes[p].L = L;
        for (int j = 0; j < L; j++) planes[p].k[j] = dirs[j];
        planes[p].in.b = B_IN;
        planes[p].in.off = p == 0 ? 0 : (long long)g.Hp * g.Wp + (long long)(p - 1) * g.Hcp * g.Wcp;
        planes[p].in.rs = planes[p].W;
        planes[p].in.cs = 1;
        planes[p].coef = f.poff[p];
    }
    return planes;
}

bool valid_params(const cvc_params* prm) {
    return prm && prm->width >= 1 && prm->height >= 1 && prm->width <= 65535 && prm->height <= 65535 &&
           valid_dirs(prm->levels, prm->dirs_log2) && prm->qph >= 1 && prm->qph <= 181 && prm->qpl >= 1 &&
           prm->qpl <= 71 && prm->subband_threshold >= 0.0f && prm->key_interval >= 1;
}

std::vector<PlaneRef> plan_planes(int h, int w, int levels, const int* dirs, int batch, long long total) {
    std::vector<PlaneRef> planes;
    for (int b = 0; b < batch; b++) {
        PlaneRef r;
        memset(&r, 0, sizeof(r));
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

}  // namespace

// ====================================================================== plan
struct cvc_ct_plan {
    int h = 0, w = 0, L = 0, k[CVC_MAX_LEVELS] = {0}, batch = 0;
    PlaneLayout lay;
    CtEngine eng;
    float* d_work = nullptr;
    std::vector<void*> allocs;
    ~cvc_ct_plan() {
        for (void* p : allocs) cudaFree(p);
    }
};

// ===================================================================== codec
struct cvc_codec {
    cvc_params prm;
    ColourGeom cg;
    PlaneLayout ly, lc;
    FrameGeom fg;
    QuantParams qp;
    StreamHeader hdr;
    long long ncoef = 0;
    int ncomp = 0;
    long long max_stream = 0;
    long long nplane = 0;   // floats of the three padded planes
    CtEngine eng;
    float *d_planes = nullptr, *d_coef = nullptr, *d_work = nullptr, *d_rplanes = nullptr, *d_dcoef = nullptr;
    int16_t *d_est[2] = {nullptr, nullptr}, *d_dst[2] = {nullptr, nullptr}, *d_res = nullptr;
    int ecur = 0, dcur = 0;
    int nrows = 0;
    long long* d_row_off = nullptr;
    int* d_row_w = nullptr;
    uint8_t* d_row_low = nullptr;
    int* d_comp_row0 = nullptr;
    uint8_t* d_comp_low = nullptr;
    long long* d_comp_elem = nullptr;
    uint32_t *d_rowcnt = nullptr, *d_rowoff = nullptr, *d_scan_tmp = nullptr;
    uint32_t max_tok = 0;
    uint32_t *d_contrib = nullptr, *d_pos = nullptr, *d_comp_tok = nullptr;
    DecInfo* d_info = nullptr;
    uint32_t *d_err = nullptr, *d_einfo = nullptr;
    uint32_t* h_pin = nullptr;
    long long enc_frame = 0, dec_next = -1;
    bool have_enc = false, have_dec = false;
    std::vector<void*> allocs;
    // stage timing (CVC_NUM_STAGES stages)
    bool timing = false;
    cudaEvent_t ev[CVC_NUM_STAGES][2] = {};
    bool ev_used[CVC_NUM_STAGES] = {};
    double t_ms[CVC_NUM_STAGES] = {};
    long long t_launches[CVC_NUM_STAGES] = {};
    ~cvc_codec() {
        for (void* p : allocs) cudaFree(p);
        if (h_pin) cudaFreeHost(h_pin);
        for (int s = 0; s < CVC_NUM_STAGES; s++)
            for (int e = 0; e < 2; e++)
                if (ev[s][e]) cudaEventDestroy(ev[s][e]);
    }
    void stage_begin(int s, cudaStream_t st) {
        if (timing) cudaEventRecord(ev[s][0], st);
    }
    void stage_end(int s, cudaStream_t st, int launches) {
        note_launches(launches);
        if (!timing) return;
        cudaEventRecord(ev[s][1], st);
        ev_used[s] = true;
        t_launches[s] += launches;
    }
    void stage_collect() {  // after a stream synchronisation
        for (int s = 0; s < CVC_NUM_STAGES; s++) {
            if (!ev_used[s]) continue;
            float ms = 0.f;
            if (cudaEventElapsedTime(&ms, ev[s][0], ev[s][1]) == cudaSuccess) t_ms[s] += ms;
            ev_used[s] = false;
        }
    }
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
    if (!valid_dirs(levels, dirs_log2)) return 0;
    return modulus(levels, dirs_log2);
}

cvc_status cvc_ct_layout(int h, int w, int levels, const int* dirs_log2, cvc_ct_layout_t* out) {
    if (!out || !valid_dirs(levels, dirs_log2)) return CVC_ERR_INVALID_ARG;
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
    if (!out) return CVC_ERR_INVALID_ARG;
    *out = nullptr;
    if (!valid_dirs(levels, dirs_log2) || batch < 1) return CVC_ERR_INVALID_ARG;
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
    std::vector<PlaneRef> planes = plan_planes(h, w, levels, dirs_log2, batch, p->lay.total);
    if (!engine_build(&p->eng, planes) || !dalloc(p->allocs, &p->d_work, (size_t)p->eng.work_elems)) {
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

// ----------------------------------------------------------------- codec
cvc_status cvc_create(const cvc_params* prm, cvc_codec** out) {
    if (!out) return CVC_ERR_INVALID_ARG;
    *out = nullptr;
    if (!valid_params(prm)) return CVC_ERR_INVALID_ARG;
    if (prm->chroma_420 != 1) return CVC_ERR_UNSUPPORTED;
    cvc_codec* c = new (std::nothrow) cvc_codec();
    if (!c) return CVC_ERR_NOMEM;
    c->prm = *prm;
    const int L = prm->levels;
    ColourGeom& g = c->cg;
    if (!codec_geometry(prm, &g) || !make_layout(g.Hp, g.Wp, L, prm->dirs_log2, &c->ly) ||
        !make_layout(g.Hcp, g.Wcp, L, prm->dirs_log2, &c->lc)) {
        delete c;
        return CVC_ERR_UNSUPPORTED;
    }
    c->ncoef = c->ly.total + 2 * c->lc.total;
    c->ncomp = (int)(c->ly.sb.size() + 2 * c->lc.sb.size());
    c->max_stream = 32 + 4LL * c->ncomp + 2LL * 2 * c->ncoef;
    c->nplane = (long long)g.Hp * g.Wp + 2LL * g.Hcp * g.Wcp;
    FrameGeom& f = c->fg;
    f.poff[0] = 0;
    f.poff[1] = c->ly.total;
    f.poff[2] = c->ly.total + c->lc.total;
    f.low_n[0] = (long long)c->ly.sb[0].h * c->ly.sb[0].w;
    f.low_n[1] = f.low_n[2] = (long long)c->lc.sb[0].h * c->lc.sb[0].w;
    f.low_w[0] = c->ly.sb[0].w;
    f.low_w[1] = f.low_w[2] = c->lc.sb[0].w;
    f.total = c->ncoef;
    c->qp.qph = (float)prm->qph;
    c->qp.qpl = (float)prm->qpl;
    c->qp.threshold = prm->subband_threshold;
    c->qp.low_scale = ldexpf(1.0f, -L);
    c->qp.qpl_denorm = ldexpf((float)prm->qpl, L);
    StreamHeader& h = c->hdr;
    memset(&h, 0, sizeof(h));
    h.levels = L;
    h.height = g.H;
    h.width = g.W;
    for (int j = 0; j < 6; j++) h.dirs[j] = j < L ? prm->dirs_log2[j] : 0;
    h.qph = prm->qph;
    h.qpl = prm->qpl;
    // transform engine over the three planes
    std::vector<PlaneRef> planes = codec_planes(g, L, prm->dirs_log2, f);
    // rows of every component in stream order
    std::vector<long long> row_off;
    std::vector<int> row_w, comp_row0;
    std::vector<uint8_t> row_low, comp_low;
    std::vector<long long> comp_elem;
    for (int p = 0; p < 3; p++) {
        const PlaneLayout& Ly = p == 0 ? c->ly : c->lc;
        for (const SubbandG& s : Ly.sb) {
            comp_row0.push_back((int)row_off.size());
            comp_low.push_back(s.kind == 0);
            comp_elem.push_back(f.poff[p] + s.off);
            for (int r = 0; r < s.h; r++) {
                row_off.push_back(f.poff[p] + s.off + (long long)r * s.w);
                row_w.push_back(s.w);
                row_low.push_back(s.kind == 0);
            }
        }
    }
    comp_row0.push_back((int)row_off.size());
    comp_elem.push_back(c->ncoef);
    c->nrows = (int)row_off.size();
    c->max_tok = (uint32_t)(2 * c->ncoef + 64);
    bool ok = engine_build(&c->eng, planes);
    auto& A = c->allocs;
    ok = ok && dalloc(A, &c->d_planes, (size_t)c->nplane) && dalloc(A, &c->d_rplanes, (size_t)c->nplane) &&
         dalloc(A, &c->d_coef, (size_t)c->ncoef) && dalloc(A, &c->d_dcoef, (size_t)c->ncoef) &&
         dalloc(A, &c->d_work, (size_t)c->eng.work_elems) && dalloc(A, &c->d_est[0], (size_t)c->ncoef) &&
         dalloc(A, &c->d_est[1], (size_t)c->ncoef) && dalloc(A, &c->d_dst[0], (size_t)c->ncoef) &&
         dalloc(A, &c->d_dst[1], (size_t)c->ncoef) && dalloc(A, &c->d_res, (size_t)c->ncoef) &&
         dalloc(A, &c->d_row_off, row_off.size()) && dalloc(A, &c->d_row_w, row_w.size()) &&
         dalloc(A, &c->d_row_low, row_low.size()) && dalloc(A, &c->d_comp_row0, comp_row0.size()) &&
         dalloc(A, &c->d_comp_low, comp_low.size()) && dalloc(A, &c->d_comp_elem, comp_elem.size()) &&
         dalloc(A, &c->d_rowcnt, (size_t)c->nrows) && dalloc(A, &c->d_rowoff, (size_t)c->nrows + 1) &&
         dalloc(A, &c->d_scan_tmp, (size_t)c->max_tok / 2048 + 8) && dalloc(A, &c->d_contrib, (size_t)c->max_tok) &&
         dalloc(A, &c->d_pos, (size_t)c->max_tok + 1) && dalloc(A, &c->d_comp_tok, (size_t)c->ncomp + 1) &&
         dalloc(A, &c->d_info, 1) && dalloc(A, &c->d_err, 1) && dalloc(A, &c->d_einfo, 4);
    ok = ok && cudaMallocHost((void**)&c->h_pin, 64) == cudaSuccess;
    ok = ok && cudaMemcpy(c->d_row_off, row_off.data(), row_off.size() * 8, cudaMemcpyHostToDevice) == cudaSuccess &&
         cudaMemcpy(c->d_row_w, row_w.data(), row_w.size() * 4, cudaMemcpyHostToDevice) == cudaSuccess &&
         cudaMemcpy(c->d_row_low, row_low.data(), row_low.size(), cudaMemcpyHostToDevice) == cudaSuccess &&
         cudaMemcpy(c->d_comp_row0, comp_row0.data(), comp_row0.size() * 4, cudaMemcpyHostToDevice) == cudaSuccess &&
         cudaMemcpy(c->d_comp_low, comp_low.data(), comp_low.size(), cudaMemcpyHostToDevice) == cudaSuccess &&
         cudaMemcpy(c->d_comp_elem, comp_elem.data(), comp_elem.size() * 8, cudaMemcpyHostToDevice) == cudaSuccess;
    ok = ok && cudaMemset(c->d_est[0], 0, (size_t)c->ncoef * 2) == cudaSuccess &&
         cudaMemset(c->d_dst[0], 0, (size_t)c->ncoef * 2) == cudaSuccess;
    if (!ok) {
        delete c;
        cudaGetLastError();
        return CVC_ERR_NOMEM;
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
    c->enc_frame = 0;
    c->dec_next = -1;
    return CVC_OK;
}

cvc_status cvc_codec_info(const cvc_codec* c, cvc_codec_info_t* out) {
    if (!c || !out) return CVC_ERR_INVALID_ARG;
    out->padded_height = c->cg.Hp;
    out->padded_width = c->cg.Wp;
    out->chroma_height = c->cg.Hc;
    out->chroma_width = c->cg.Wc;
    out->padded_chroma_height = c->cg.Hcp;
    out->padded_chroma_width = c->cg.Wcp;
    out->coeffs = c->ncoef;
    out->components = c->ncomp;
    out->max_stream_bytes = c->max_stream;
    return CVC_OK;
}

cvc_status cvc_encode_frame(cvc_codec* c, const uint8_t* d_rgb, size_t pitch_bytes, uint8_t* d_out, size_t out_cap,
                            size_t* out_len, int* frame_type, cvc_stream_t stream) {
    if (!c || !d_rgb || !d_out || !out_len || pitch_bytes < (size_t)c->cg.W * 3 || ((uintptr_t)d_out & 3))
        return CVC_ERR_INVALID_ARG;
    cudaStream_t st = (cudaStream_t)stream;
    const int type = (c->enc_frame % c->prm.key_interval) == 0 ? 0 : 1;
    const long long hdr_bytes = 32 + 4LL * c->ncomp;
    const bool hdr_fits = (long long)out_cap >= hdr_bytes;
    const long long cap_tok = hdr_fits ? ((long long)out_cap - hdr_bytes) / 2 : 0;
    float* Yp = c->d_planes;
    float* Cop = Yp + (long long)c->cg.Hp * c->cg.Wp;
    float* Cgp = Cop + (long long)c->cg.Hcp * c->cg.Wcp;
    Bases B;
    memset(&B, 0, sizeof(B));
    B.p[B_IN] = c->d_planes;
    B.p[B_COEF] = c->d_coef;
    B.p[B_WORK] = c->d_work;
    cudaMemsetAsync(c->d_err, 0, 4, st);
    // S1-S3: colour, 4:2:0, padding
    c->stage_begin(0, st);
    k_colour_fwd<<<grid_for(c->nplane), 256, 0, st>>>(d_rgb, (long long)pitch_bytes, c->cg, Yp, Cop, Cgp);
    c->stage_end(0, st, 1);
    // S4: LP analysis, S5: DFB analysis
    c->stage_begin(1, st);
    if (engine_run_part(&c->eng, FWD, 0, B, st) != cudaSuccess) return CVC_ERR_CUDA;
    c->stage_end(1, st, 0);
    c->stage_begin(2, st);
    if (engine_run_part(&c->eng, FWD, 1, B, st) != cudaSuccess) return CVC_ERR_CUDA;
    c->stage_end(2, st, 0);
    if (c->timing) {
        c->t_launches[1] += engine_part_launches(&c->eng, FWD, 0);
        c->t_launches[2] += engine_part_launches(&c->eng, FWD, 1);
    }
    // S6-S8: normalise, threshold, quantise, K/P differencing
    int16_t* qnew = c->d_est[1 - c->ecur];
    c->stage_begin(3, st);
    k_quant<<<grid_for(c->ncoef), 256, 0, st>>>(c->d_coef, c->d_est[c->ecur], c->fg, c->qp, type == 0, qnew, c->d_res,
                                                c->d_err);
    c->stage_end(3, st, 1);
    // S9: RLE rows -> bitstream
    RowTable rt{c->d_row_off, c->d_row_w, c->d_row_low, c->nrows};
    const int rows_per_block = 8;
    const int rgrid = (c->nrows + rows_per_block - 1) / rows_per_block;
    c->stage_begin(4, st);
    k_rle_count<<<rgrid, 32 * rows_per_block, 0, st>>>(c->d_res, rt, type == 0, c->d_rowcnt);
    exclusive_scan(c->d_rowcnt, (uint32_t)c->nrows, c->d_rowoff, c->d_scan_tmp, st);
    int nl = 4;
    if (hdr_fits) {
        k_rle_write<<<rgrid, 32 * rows_per_block, 0, st>>>(c->d_res, rt, type == 0, c->d_rowoff, d_out + hdr_bytes,
                                                           (uint32_t)std::min<long long>(cap_tok, 0xFFFFFFFFLL),
                                                           c->d_err);
        StreamHeader h = c->hdr;
        h.type = type;
        h.frame_index = (uint32_t)c->enc_frame;
        k_stream_header<<<(c->ncomp + 255) / 256, 256, 0, st>>>(h, c->d_rowoff, c->d_comp_row0, c->ncomp, d_out,
                                                                c->d_einfo);
        nl += 2;
    } else {
        cudaMemcpyAsync(c->d_einfo, c->d_rowoff + c->nrows, 4, cudaMemcpyDeviceToDevice, st);
    }
    c->stage_end(4, st, nl);
    cudaMemcpyAsync(c->h_pin, c->d_err, 4, cudaMemcpyDeviceToHost, st);
    cudaMemcpyAsync(c->h_pin + 1, c->d_einfo, 4, cudaMemcpyDeviceToHost, st);
    if (cudaStreamSynchronize(st) != cudaSuccess || cudaGetLastError() != cudaSuccess) return CVC_ERR_CUDA;
    c->stage_collect();
    const uint32_t err = c->h_pin[0];
    const long long need = hdr_bytes + 2LL * c->h_pin[1];
    *out_len = (size_t)need;
    if (frame_type) *frame_type = type;
    if (err & EF_OVERFLOW) return CVC_ERR_OVERFLOW;
    if (!hdr_fits || need > (long long)out_cap || (err & EF_CAPACITY)) return CVC_ERR_CAPACITY;
    c->ecur = 1 - c->ecur;
    c->enc_frame += 1;
    c->have_enc = true;
    return CVC_OK;
}

cvc_status cvc_decode_frame(cvc_codec* c, const uint8_t* d_in, size_t in_len, uint8_t* d_rgb, size_t pitch_bytes,
                            cvc_stream_t stream) {
    if (!c || !d_in || !d_rgb || pitch_bytes < (size_t)c->cg.W * 3) return CVC_ERR_INVALID_ARG;
    cudaStream_t st = (cudaStream_t)stream;
    const long long hdr_bytes = 32 + 4LL * c->ncomp;
    long long avail = ((long long)in_len - hdr_bytes) / 2;
    uint32_t max_tok = (uint32_t)std::max(0LL, std::min<long long>(avail, c->max_tok));
    cudaMemsetAsync(c->d_err, 0, 4, st);
    // bitstream parse and run-length expansion
    c->stage_begin(5, st);
    k_dec_parse<<<1, 1024, 0, st>>>(d_in, (long long)in_len, c->hdr, c->ncomp, c->dec_next, max_tok, c->d_comp_tok,
                                    c->d_info, c->d_err);
    const uint8_t* tok = d_in + hdr_bytes;
    k_dec_contrib<<<grid_for(max_tok), 256, 0, st>>>(tok, c->d_comp_tok, c->ncomp, c->d_comp_low, c->d_info,
                                                     c->d_contrib, max_tok, c->d_err);
    exclusive_scan(c->d_contrib, max_tok, c->d_pos, c->d_scan_tmp, st);
    k_dec_check<<<(c->ncomp + 256) / 256, 256, 0, st>>>(c->d_comp_tok, c->d_pos, c->d_comp_elem, c->ncomp, c->d_info,
                                                        c->d_err);
    cudaMemsetAsync(c->d_res, 0, (size_t)c->ncoef * 2, st);
    k_dec_scatter<<<grid_for(max_tok), 256, 0, st>>>(tok, c->d_comp_tok, c->ncomp, c->d_comp_low, c->d_info, c->d_pos,
                                                     c->ncoef, c->d_res);
    c->stage_end(5, st, 7);
    // inverse K/P differencing and dequantisation
    int16_t* qnew = c->d_dst[1 - c->dcur];
    c->stage_begin(6, st);
    k_unquant<<<grid_for(c->ncoef), 256, 0, st>>>(c->d_res, c->d_dst[c->dcur], c->fg, c->qp, c->d_info, qnew,
                                                  c->d_dcoef);
    const int lowcols = c->fg.low_w[0] + 2 * c->fg.low_w[1];
    k_unquant_keylow<<<(lowcols + 255) / 256, 256, 0, st>>>(c->d_res, c->fg, c->qp, c->d_info, qnew, c->d_dcoef);
    c->stage_end(6, st, 2);
    // inverse transform: DFB synthesis, then LP synthesis
    Bases B;
    memset(&B, 0, sizeof(B));
    B.p[B_COEF] = c->d_dcoef;
    B.p[B_WORK] = c->d_work;
    B.p[B_OUT] = c->d_rplanes;
    c->stage_begin(7, st);
    if (engine_run_part(&c->eng, INV, 1, B, st) != cudaSuccess) return CVC_ERR_CUDA;
    c->stage_end(7, st, 0);
    c->stage_begin(8, st);
    if (engine_run_part(&c->eng, INV, 0, B, st) != cudaSuccess) return CVC_ERR_CUDA;
    c->stage_end(8, st, 0);
    if (c->timing) {
        c->t_launches[7] += engine_part_launches(&c->eng, INV, 1);
        c->t_launches[8] += engine_part_launches(&c->eng, INV, 0);
    }
    // rounding, chroma upsampling, inverse colour transform
    float* Yp = c->d_rplanes;
    float* Cop = Yp + (long long)c->cg.Hp * c->cg.Wp;
    float* Cgp = Cop + (long long)c->cg.Hcp * c->cg.Wcp;
    c->stage_begin(9, st);
    k_colour_inv<<<grid_for((long long)c->cg.H * c->cg.W), 256, 0, st>>>(Yp, Cop, Cgp, c->cg, d_rgb,
                                                                         (long long)pitch_bytes);
    c->stage_end(9, st, 1);
    cudaMemcpyAsync(c->h_pin, c->d_err, 4, cudaMemcpyDeviceToHost, st);
    cudaMemcpyAsync(c->h_pin + 2, c->d_info, sizeof(DecInfo), cudaMemcpyDeviceToHost, st);
    if (cudaStreamSynchronize(st) != cudaSuccess || cudaGetLastError() != cudaSuccess) return CVC_ERR_CUDA;
    c->stage_collect();
    const uint32_t err = c->h_pin[0];
    DecInfo info;
    memcpy(&info, c->h_pin + 2, sizeof(info));
    if (err & EF_STATE) return CVC_ERR_STATE;
    if (err & (EF_CORRUPT | EF_MISMATCH)) return CVC_ERR_CORRUPT;
    c->dcur = 1 - c->dcur;
    c->dec_next = (long long)info.frame_index + 1;
    c->have_dec = true;
    return CVC_OK;
}

cvc_status cvc_codec_set_timing(cvc_codec* c, int on) {
    if (!c) return CVC_ERR_INVALID_ARG;
    if (on) {
        for (int s = 0; s < CVC_NUM_STAGES; s++) {
            for (int e = 0; e < 2; e++)
                if (!c->ev[s][e] && cudaEventCreate(&c->ev[s][e]) != cudaSuccess) return CVC_ERR_CUDA;
            c->t_ms[s] = 0.0;
            c->t_launches[s] = 0;
            c->ev_used[s] = false;
        }
    }
    c->timing = on != 0;
    return CVC_OK;
}

cvc_status cvc_codec_timing(const cvc_codec* c, double* ms, long long* launches) {
    if (!c) return CVC_ERR_INVALID_ARG;
    for (int s = 0; s < CVC_NUM_STAGES; s++) {
        if (ms) ms[s] = c->t_ms[s];
        if (launches) launches[s] = c->t_launches[s];
    }
    return CVC_OK;
}

unsigned long long cvc_kernel_launches(void) { return g_launches.load(); }

cvc_status cvc_debug_plan_tables(const cvc_params* params, int h, int w, int levels, const int* dirs_log2, int batch,
                                 int mode, void* buf, size_t cap, size_t* used) {
    if (!used || mode < 0 || mode > 3) return CVC_ERR_INVALID_ARG;
    std::vector<PlaneRef> planes;
    unsigned long long elems[4] = {0, 0, 0, 0};
    if (params) {
        if (!valid_params(params)) return CVC_ERR_INVALID_ARG;
        ColourGeom g;
        PlaneLayout ly, lc;
        if (!codec_geometry(params, &g) || !make_layout(g.Hp, g.Wp, params->levels, params->dirs_log2, &ly) ||
            !make_layout(g.Hcp, g.Wcp, params->levels, params->dirs_log2, &lc))
            return CVC_ERR_UNSUPPORTED;
        FrameGeom f;
        memset(&f, 0, sizeof(f));
        f.poff[1] = ly.total;
        f.poff[2] = ly.total + lc.total;
        planes = codec_planes(g, params->levels, params->dirs_log2, f);
        elems[0] = elems[3] = (unsigned long long)g.Hp * g.Wp + 2ULL * g.Hcp * g.Wcp;
        elems[1] = (unsigned long long)(ly.total + 2 * lc.total);
    } else {
        PlaneLayout lay;
        if (!valid_dirs(levels, dirs_log2) || batch < 1 || !make_layout(h, w, levels, dirs_log2, &lay))
            return CVC_ERR_INVALID_ARG;
        planes = plan_planes(h, w, levels, dirs_log2, batch, lay.total);
        elems[0] = elems[3] = (unsigned long long)batch * h * w;
        elems[1] = (unsigned long long)batch * lay.total;
    }
    CtEngine e;
    if (!engine_build(&e, planes, false)) return CVC_ERR_INVALID_ARG;
    elems[2] = (unsigned long long)e.work_elems;
    // launch order of the mode
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
    if (analysis) { push_lp(); push_dfb(); }
    else { push_dfb(); push_lp(); }
    size_t need = 24 + 32;
    for (const Item& it : items) need += 8 + it.n * it.sz;
    *used = need;
    if (!buf || cap < need) return CVC_ERR_CAPACITY;
    uint8_t* o = (uint8_t*)buf;
    uint32_t hdr[6] = {0x43564350u, (uint32_t)items.size(), (uint32_t)sizeof(LpJob), (uint32_t)sizeof(DfbAJob),
                       (uint32_t)sizeof(DfbBJob), 0u};
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
    return CVC_OK;
}

cvc_status cvc_codec_inspect(const cvc_codec* c, int which, float* d_out, size_t cap_elems, cvc_stream_t stream) {
    if (!c || !d_out || which < 0 || which > 2) return CVC_ERR_INVALID_ARG;
    const float* src = which == 0 ? c->d_planes : (which == 1 ? c->d_coef : c->d_rplanes);
    size_t n = (size_t)(which == 1 ? c->ncoef : c->nplane);
    if (cap_elems < n) return CVC_ERR_INVALID_ARG;
    return cudaMemcpyAsync(d_out, src, n * 4, cudaMemcpyDeviceToDevice, (cudaStream_t)stream) == cudaSuccess
               ? CVC_OK
               : CVC_ERR_CUDA;
}

}  // extern "C"
