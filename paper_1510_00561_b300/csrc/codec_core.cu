// codec_core.cu -- host side of the multi-stream codec core: per-stream
// descriptors, block maps, row and component tables, one device arena, the
// fixed launch sequence of a step and its CUDA-graph capture.
#include <algorithm>
#include <cstring>

#include "codec_core.cuh"

namespace cvc {

namespace {

inline int round_up(int v, int m) { return (v + m - 1) / m * m; }
inline long long cdiv(long long a, long long b) { return (a + b - 1) / b; }

// carves one allocation into aligned sub-buffers
struct Carve {
    std::vector<std::pair<void**, size_t>> items;
    size_t total = 0;
    template <class T>
    void add(T** p, size_t n) {
        total = (total + 255) & ~size_t(255);
        items.push_back({reinterpret_cast<void**>(p), total});
        total += std::max<size_t>(n, 1) * sizeof(T);
    }
    void assign(char* base) {
        for (auto& it : items) *it.first = base + it.second;
    }
};

void carve_all(Core* c, Carve& k) {
    const size_t n = (size_t)c->n;
    k.add(&c->d_sd, n);
    k.add(&c->d_sc, n);
    k.add(&c->d_rs, n);
    k.add(&c->d_ctl, n);
    k.add(&c->d_pd, c->h_pd.size());
    k.add(&c->d_blk_colour, c->h_blk_colour.size());
    k.add(&c->d_blk_plane, c->h_blk_plane.size());
    k.add(&c->d_row_off, c->h_row_off.size());
    k.add(&c->d_row_w, c->h_row_w.size());
    k.add(&c->d_row_stream, c->h_row_stream.size());
    k.add(&c->d_row_comp, c->h_row_comp.size());
    k.add(&c->d_row_mc, c->h_row_mc.size());
    k.add(&c->d_row_low, c->h_row_low.size());
    k.add(&c->d_comp_tile0, c->h_comp_tile0.size());
    k.add(&c->d_tile_off, c->h_tile_off.size());
    k.add(&c->d_tile_n, c->h_tile_n.size());
    k.add(&c->d_tile_w, c->h_tile_w.size());
    k.add(&c->d_tile_stream, c->h_tile_stream.size());
    k.add(&c->d_tile_low, c->h_tile_low.size());
    k.add(&c->d_comp_stream, c->h_comp_stream.size());
    k.add(&c->d_comp_low, c->h_comp_low.size());
    k.add(&c->d_comp_level, c->h_comp_level.size());
    k.add(&c->d_comp_plane, c->h_comp_plane.size());
    k.add(&c->d_comp_ey, c->h_comp_ey.size());
    k.add(&c->d_comp_ex, c->h_comp_ex.size());
    k.add(&c->d_blk_motion, c->h_blk_motion.size());
    k.add(&c->d_luma[0], (size_t)c->luma_total);
    k.add(&c->d_luma[1], (size_t)c->luma_total);
    k.add(&c->d_mv, 2 * (size_t)c->mv_pairs);
    k.add(&c->d_comp_elem, c->h_comp_elem.size());
    k.add(&c->d_planes, (size_t)c->nplane);
    k.add(&c->d_rplanes, (size_t)c->nplane);
    k.add(&c->d_coef, (size_t)c->ncoef);
    k.add(&c->d_dcoef, (size_t)c->ncoef);
    // the sub-pyramids of every decoding scale fit in the full transform's workspace
    long long work = c->eng.work_elems;
    for (const auto& sp : c->scale) work = std::max(work, sp->eng.work_elems);
    k.add(&c->d_work, (size_t)work);
    for (const auto& sp : c->scale) {
        k.add(&sp->d_desc, n);
        k.add(&sp->d_blk, sp->h_blk.size());
    }
    for (int b = 0; b < 2; b++) {
        k.add(&c->d_est_buf[b], (size_t)c->ncoef);
        k.add(&c->d_dst_buf[b], (size_t)c->ncoef);
    }
    k.add(&c->d_res, (size_t)c->ncoef + 8);   // the RLE reads whole 16-byte chunks
    k.add(&c->d_tilecnt, (size_t)c->ntiles);
    k.add(&c->d_tileoff, (size_t)c->ntiles + 1);
    k.add(&c->d_scan_tmp, (size_t)cdiv(c->ntiles, 2048) + 8);
    k.add(&c->d_comp_tok, (size_t)c->ncomp);
    k.add(&c->d_tok_base, n + 1);
    k.add(&c->d_dtile_base, n + 1);
    k.add(&c->d_dtile_sum, (size_t)c->max_dtiles);
    k.add(&c->d_dtile_pre, (size_t)c->max_dtiles + 1);
    k.add(&c->d_comp_codes, (size_t)c->ncomp);
    k.add(&c->d_scan_tmp2, 1024 + 8);
}

size_t engine_table_bytes_of(const CtEngine& e) {
    size_t b = 0;
    for (int m = 0; m < 4; m++) {
        for (const LaunchLp& L : e.lp[m]) b += L.njobs * sizeof(LpJob) + (size_t)L.nblocks * sizeof(int) + 1024;
        for (const LaunchDfb& L : e.dfb[m])
            b += L.njobs * (L.kind == 0 ? sizeof(DfbAJob) : sizeof(DfbBJob)) + (size_t)L.nblocks * sizeof(int) + 1024;
        for (const TailTables& T : e.h_tail[m])
            b += T.planes.size() * sizeof(TailPlane) + T.steps.size() * sizeof(TailStep) +
                 T.lp.size() * sizeof(LpJob) + T.a.size() * sizeof(DfbAJob) + T.b.size() * sizeof(DfbBJob) + 5 * 1024;
    }
    return b;
}

size_t engine_table_bytes(const Core* c) {
    size_t b = engine_table_bytes_of(c->eng);
    for (const auto& sp : c->scale) b += engine_table_bytes_of(sp->eng);
    return b;
}

// the decoder back end of every scale 0 .. max_levels (host tables; see ScalePlan)
cvc_status plan_scales(Core* c) {
    c->scale.clear();
    for (int sc = 0; sc <= c->max_levels; sc++) {
        std::unique_ptr<ScalePlan> sp(new ScalePlan());
        sp->h_desc.assign((size_t)c->n, ScaleDesc{});
        std::vector<PlaneRef> sub;
        for (int s = 0; s < c->n; s++) {
            const cvc_params& P = c->prm[s];
            if (P.levels < sc) continue;
            const SDesc& D = c->sd[s];
            const ColourGeom& g = D.cg;
            const int f = 1 << sc;
            ScaleDesc& Q = sp->h_desc[s];
            Q.H = (g.H + f - 1) >> sc;
            Q.W = (g.W + f - 1) >> sc;
            Q.Hc = (g.Hc + f - 1) >> sc;
            Q.Wc = (g.Wc + f - 1) >> sc;
            Q.norm = ldexpf(1.0f, -sc);
            Q.st8 = D.qp.st8;
            Q.blk0 = (int)sp->h_blk.size();
            // padded planes are multiples of 2^L, so these sizes are exact
            const int hs[3] = {g.Hp >> sc, g.Hcp >> sc, g.Hcp >> sc}, ws[3] = {g.Wp >> sc, g.Wcp >> sc, g.Wcp >> sc};
            Q.rs_y = ws[0];
            Q.rs_c = ws[1];
            const PlaneLayout* lays[3] = {&c->ly[s], &c->lc[s], &c->lc[s]};
            const long long poff[3] = {D.coef_off, D.coef_off + c->ly[s].total,
                                       D.coef_off + c->ly[s].total + c->lc[s].total};
            if (sc == P.levels) {
                // no level left: the lowpass bands ((H >> L) x (W >> L), dequantised) are the planes
                Q.src = 1;
                for (int p = 0; p < 3; p++) Q.off[p] = poff[p] + lays[p]->sb[0].off;
            } else {
                Q.src = 0;
                Q.off[0] = D.plane_off;
                Q.off[1] = Q.off[0] + (long long)hs[0] * ws[0];
                Q.off[2] = Q.off[1] + (long long)hs[1] * ws[1];
            }
            if (sc > 0 && sc < P.levels) {
                // subbands of levels sc+1..L sit in the layout in the order of the
                // sub-pyramid's own layout, right after the lowpass: shifting the
                // coefficient base by (first subband of level sc+1) - (lowpass size)
                // lines them up; the lowpass keeps its own offset
                int first = 1;
                for (int j = 0; j < sc; j++) first += 1 << P.dirs_log2[j];
                for (int p = 0; p < 3; p++) {
                    const PlaneLayout& Lp = *lays[p];
                    const long long nlow = (long long)Lp.sb[0].h * Lp.sb[0].w;
                    PlaneRef r;
                    memset(&r, 0, sizeof(r));
                    r.H = hs[p];
                    r.W = ws[p];
                    r.L = P.levels - sc;
                    for (int j = 0; j < r.L; j++) r.k[j] = P.dirs_log2[sc + j];
                    r.in.b = B_OUT;
                    r.in.off = Q.off[p];
                    r.in.rs = ws[p];
                    r.in.cs = 1;
                    r.coef = poff[p] + Lp.sb[first].off - nlow;
                    r.low_coef = poff[p] + Lp.sb[0].off;
                    r.taps = P.dfb_taps;
                    r.stream = s;
                    sub.push_back(r);
                }
            }
            if ((long long)sp->h_blk.size() + Q.H > (1LL << 30)) return CVC_ERR_UNSUPPORTED;
            sp->h_blk.insert(sp->h_blk.end(), (size_t)Q.H, s);
        }
        if (sc > 0 && !engine_build(&sp->eng, sub, false)) return CVC_ERR_UNSUPPORTED;
        c->scale.push_back(std::move(sp));
    }
    return CVC_OK;
}

template <class T>
bool put(T* d, const std::vector<T>& h) {
    if (h.empty()) return true;
    return cudaMemcpy(d, h.data(), h.size() * sizeof(T), cudaMemcpyHostToDevice) == cudaSuccess;
}

}  // namespace

bool dirs_valid(int levels, const int* dirs) {
    if (levels < 1 || levels > CVC_MAX_LEVELS || !dirs) return false;
    for (int j = 0; j < levels; j++)
        if (dirs[j] < 0 || dirs[j] > CVC_MAX_DIRS_LOG2) return false;
    return true;
}

bool codec_params_valid(const cvc_params* prm) {
    return prm && prm->width >= 1 && prm->height >= 1 && prm->width <= 65535 && prm->height <= 65535 &&
           dirs_valid(prm->levels, prm->dirs_log2) && prm->qph >= 1 && prm->qph <= 181 && prm->qpl >= 1 &&
           prm->qpl <= 71 && prm->subband_threshold >= 0.0f && prm->key_interval >= 1 && prm->motion_range >= 0 &&
           prm->motion_range <= CVC_MAX_MOTION_RANGE && (prm->storage8 == 0 || prm->storage8 == 1) &&
           (prm->dfb_taps == 0 || prm->dfb_taps == 4 || prm->dfb_taps == 6 || prm->dfb_taps == 8);
}

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

std::vector<PlaneRef> codec_planes(const ColourGeom& g, int L, const int* dirs, int taps, long long plane_off,
                                   const long long poff[3], int stream) {
    std::vector<PlaneRef> planes(3);
    for (int p = 0; p < 3; p++) {
        memset(&planes[p], 0, sizeof(PlaneRef));
        planes[p].low_coef = -1;
        planes[p].stream = stream;
        planes[p].H = p == 0 ? g.Hp : g.Hcp;
        planes[p].W = p == 0 ? g.Wp : g.Wcp;
        planes[p].L = L;
        for (int j = 0; j < L; j++) planes[p].k[j] = dirs[j];
        planes[p].in.b = B_IN;
        planes[p].in.off =
            plane_off + (p == 0 ? 0 : (long long)g.Hp * g.Wp + (long long)(p - 1) * g.Hcp * g.Wcp);
        planes[p].in.rs = planes[p].W;
        planes[p].in.cs = 1;
        planes[p].coef = poff[p];
        planes[p].taps = taps;
    }
    return planes;
}

ScalePlan::~ScalePlan() {
    for (int m = 0; m < 4; m++)
        if (gexec[m]) cudaGraphExecDestroy(gexec[m]);
}

Core::~Core() {
    scale.clear();   // graphs first
    if (cap_stream) cudaStreamDestroy(cap_stream);
    if (side) cudaStreamDestroy(side);
    for (int k = 0; k < 2; k++) {
        if (ev_fork[k]) cudaEventDestroy(ev_fork[k]);
        if (ev_join[k]) cudaEventDestroy(ev_join[k]);
    }
    if (arena) cudaFree(arena);
    for (int k = 0; k < CORE_RING; k++) {
        if (ring_sc[k]) cudaFreeHost(ring_sc[k]);
        if (ring_rs[k]) cudaFreeHost(ring_rs[k]);
        if (ring_ev[k]) cudaEventDestroy(ring_ev[k]);
    }
    for (int s = 0; s < CVC_NUM_STAGES; s++)
        for (int e = 0; e < 2; e++)
            if (ev[s][e]) cudaEventDestroy(ev[s][e]);
}

cvc_status core_plan(Core* c, const cvc_params* params, int n) {
    if (!params || n < 1) return CVC_ERR_INVALID_ARG;
    for (int s = 0; s < n; s++)
        if (!codec_params_valid(&params[s])) return CVC_ERR_INVALID_ARG;
    for (int s = 0; s < n; s++)
        if (params[s].chroma_420 != 1) return CVC_ERR_UNSUPPORTED;
    c->n = n;
    c->prm.assign(params, params + n);
    c->sd.assign(n, SDesc{});
    c->ly.assign(n, PlaneLayout{});
    c->lc.assign(n, PlaneLayout{});
    std::vector<PlaneRef> planes;
    long long plane_off = 0, coef_off = 0, sum_tok = 0;
    for (int s = 0; s < n; s++) {
        const cvc_params& P = params[s];
        SDesc& D = c->sd[s];
        memset(&D, 0, sizeof(D));
        const int L = P.levels;
        ColourGeom& g = D.cg;
        if (!codec_geometry(&P, &g) || !make_layout(g.Hp, g.Wp, L, P.dirs_log2, &c->ly[s]) ||
            !make_layout(g.Hcp, g.Wcp, L, P.dirs_log2, &c->lc[s]))
            return CVC_ERR_UNSUPPORTED;
        const PlaneLayout& Ly = c->ly[s];
        const PlaneLayout& Lc = c->lc[s];
        D.qp.qph = (float)P.qph;
        D.qp.qpl = (float)P.qpl;
        D.qp.threshold = P.subband_threshold;
        D.qp.low_scale = ldexpf(1.0f, -L);
        D.qp.qpl_denorm = ldexpf((float)P.qpl, L);
        D.qp.st8 = P.storage8;
        D.qp.rqph = (P.qph & (P.qph - 1)) == 0 ? 1.0f / (float)P.qph : 0.0f;
        D.qp.rqpl = (P.qpl & (P.qpl - 1)) == 0 ? 1.0f / (float)P.qpl : 0.0f;
        if (D.qp.rqph == 0.0f || D.qp.rqpl == 0.0f) c->quant_pow2 = false;
        D.hdr.levels = L;
        D.hdr.height = g.H;
        D.hdr.width = g.W;
        for (int j = 0; j < 6; j++) D.hdr.dirs[j] = j < L ? P.dirs_log2[j] : 0;
        D.hdr.qph = P.qph;
        D.hdr.qpl = P.qpl;
        D.hdr.flags = P.storage8 | (((P.dfb_taps ? P.dfb_taps : 4) / 2 - 2) << 1);
        D.plane_off = plane_off;
        D.nplane = (long long)g.Hp * g.Wp + 2LL * g.Hcp * g.Wcp;
        D.coef_off = coef_off;
        D.ncoef = Ly.total + 2 * Lc.total;
        D.row0 = (int)c->h_row_off.size();
        D.tile0 = (int)c->h_tile_off.size();
        D.comp0 = (int)c->h_comp_low.size();
        D.ncomp = (int)(Ly.sb.size() + 2 * Lc.sb.size());
        D.hdr_bytes = 32 + 4LL * D.ncomp;
        D.max_tok = 2 * D.ncoef + 64;
        D.mv_range = P.motion_range;
        D.key_interval = P.key_interval;
        if (P.motion_range > 0) {
            // 16 x 16 blocks of the padded luma plane, one motion search block each
            D.nby = (g.Hp + 15) / 16;
            D.nbx = (g.Wp + 15) / 16;
            D.mv_bytes = 2LL * D.nby * D.nbx;
            D.mv_off = c->mv_pairs;
            D.luma_off = c->luma_total;
            D.blk_motion = (int)c->h_blk_motion.size();
            c->mv_pairs += (long long)D.nby * D.nbx;
            c->luma_total += (long long)g.Hp * g.Wp;
            if ((long long)c->h_blk_motion.size() + D.nby * D.nbx > (1LL << 30)) return CVC_ERR_UNSUPPORTED;
            c->h_blk_motion.insert(c->h_blk_motion.end(), (size_t)D.nby * D.nbx, s);
            // 128 threads walk the candidates in groups of four displacements
            c->motion_threads = 128;
            c->motion_rmax = std::max(c->motion_rmax, P.motion_range);
            c->motion_ws = (16 + 2 * c->motion_rmax + 4 + 3) & ~3;   // word reads: a multiple of 4
            c->motion_smem = (16 + 2 * c->motion_rmax) * c->motion_ws;
        }
        D.blk_colour = (int)c->h_blk_colour.size();
        // forward colour kernel: one block per padded luma row and per padded chroma row
        // (the inverse one, per output row, is planned per decoding scale)
        const long long nb_col = (long long)g.Hp + g.Hcp;
        if ((long long)c->h_blk_colour.size() + nb_col > (1LL << 30)) return CVC_ERR_UNSUPPORTED;
        c->h_blk_colour.insert(c->h_blk_colour.end(), (size_t)nb_col, s);
        const long long poff[3] = {coef_off, coef_off + Ly.total, coef_off + Ly.total + Lc.total};
        for (int p = 0; p < 3; p++) {
            const PlaneLayout& Lp = p == 0 ? Ly : Lc;
            // levels 1..d follow the lowpass in the layout
            D.pstart[p] = poff[p] - coef_off;
            D.nlow[p] = (long long)Lp.sb[0].h * Lp.sb[0].w;
            for (int d = 0; d <= CVC_MAX_LEVELS; d++) {
                long long a = 0;
                for (const SubbandG& sb : Lp.sb)
                    if (sb.kind != 0 && sb.level <= d) a += (long long)sb.h * sb.w;
                D.absent[d][p] = a;
            }
            PDesc pd;
            memset(&pd, 0, sizeof(pd));
            pd.coef_off = poff[p];
            pd.total = Lp.total;
            pd.low_n = (long long)Lp.sb[0].h * Lp.sb[0].w;
            pd.low_w = Lp.sb[0].w;
            pd.stream = s;
            pd.first_block = (int)c->h_blk_plane.size();
            const long long nb = cdiv(Lp.total, ELEM_BLOCK);
            if ((long long)c->h_blk_plane.size() + nb > (1LL << 30)) return CVC_ERR_UNSUPPORTED;
            c->h_blk_plane.insert(c->h_blk_plane.end(), (size_t)nb, (int)c->h_pd.size());
            c->h_pd.push_back(pd);
            c->lowcols += pd.low_w;
            // rows of every component, in stream order
            for (const SubbandG& sb : Lp.sb) {
                const int comp = (int)c->h_comp_low.size();
                c->h_comp_tile0.push_back((int)c->h_tile_off.size());
                c->h_comp_low.push_back(sb.kind == 0);
                c->h_comp_level.push_back((uint8_t)sb.level);
                c->h_comp_plane.push_back((uint8_t)p);
                // luma samples per element: the plane's size over the component's, doubled for chroma
                int ey = p > 0, ex = p > 0;
                while (((p == 0 ? g.Hp : g.Hcp) >> (ey - (p > 0))) > sb.h) ey++;
                while (((p == 0 ? g.Wp : g.Wcp) >> (ex - (p > 0))) > sb.w) ex++;
                c->h_comp_ey.push_back((uint8_t)ey);
                c->h_comp_ex.push_back((uint8_t)ex);
                c->h_comp_stream.push_back(s);
                c->h_comp_elem.push_back(poff[p] - coef_off + sb.off);
                const int rpt = std::max(1, RLE_TILE / sb.w);   // rows per RLE tile
                for (int r = 0; r < sb.h; r += rpt) {
                    c->h_tile_off.push_back(poff[p] + sb.off + (long long)r * sb.w);
                    c->h_tile_n.push_back(std::min(rpt, sb.h - r) * sb.w);
                    c->h_tile_w.push_back(sb.w);
                    c->h_tile_stream.push_back(s);
                    c->h_tile_low.push_back(sb.kind == 0);
                }
                for (int r = 0; r < sb.h; r++) {
                    c->h_row_off.push_back(poff[p] + sb.off + (long long)r * sb.w);
                    c->h_row_w.push_back(sb.w);
                    c->h_row_low.push_back(sb.kind == 0);
                    c->h_row_stream.push_back(s);
                    c->h_row_comp.push_back(comp);
                    c->h_row_mc.push_back(make_int4(r, sb.h, ey, ex));
                }
            }
        }
        D.nrows = (int)c->h_row_off.size() - D.row0;
        D.ntiles = (int)c->h_tile_off.size() - D.tile0;
        std::vector<PlaneRef> sp = codec_planes(g, L, P.dirs_log2, P.dfb_taps, plane_off, poff, s);
        planes.insert(planes.end(), sp.begin(), sp.end());
        plane_off += D.nplane;
        coef_off += D.ncoef;
        sum_tok += D.max_tok;
        c->max_dtiles += cdiv(D.max_tok, DEC_TILE);
        if (D.ncomp > DEC_MAX_COMP) return CVC_ERR_UNSUPPORTED;
    }
    c->h_comp_tile0.push_back((int)c->h_tile_off.size());   // sentinel: end of the last component
    c->nplane = plane_off;
    c->ncoef = coef_off;
    c->sum_max_tok = sum_tok;
    c->nrows = (int)c->h_row_off.size();
    c->ntiles = (int)c->h_tile_off.size();
    c->ncomp = (int)c->h_comp_low.size();
    c->nplanes = (int)c->h_pd.size();
    // token positions and element offsets are 32-bit on the device
    if (sum_tok > 0xFFFFFF00LL || c->ncoef > 0x7FFFFFFFLL) return CVC_ERR_UNSUPPORTED;
    if (!engine_build(&c->eng, planes, false)) return CVC_ERR_UNSUPPORTED;
    c->max_levels = 0;
    for (int s = 0; s < n; s++) c->max_levels = std::max(c->max_levels, params[s].levels);
    return plan_scales(c);
}

size_t core_device_bytes(const Core* c) {
    // carve_all records where each member pointer will point; nothing is written through them here
    Carve k;
    carve_all(const_cast<Core*>(c), k);
    return k.total + engine_table_bytes(c);
}

cvc_status core_alloc(Core* c) {
    // the same job tables again, now uploaded
    const std::vector<PlaneRef> planes = c->eng.planes;
    if (!engine_build(&c->eng, planes, true)) {
        cudaGetLastError();
        return CVC_ERR_NOMEM;
    }
    for (size_t sc = 1; sc < c->scale.size(); sc++) {
        CtEngine& e = c->scale[sc]->eng;
        const std::vector<PlaneRef> sub = e.planes;
        if (!engine_build(&e, sub, true)) {
            cudaGetLastError();
            return CVC_ERR_NOMEM;
        }
    }
    if (lp_prepare() != cudaSuccess || dfb_prepare() != cudaSuccess || tail_prepare() != cudaSuccess)
        return CVC_ERR_CUDA;
    Carve k;
    carve_all(c, k);
    c->arena_bytes = k.total;
    if (cudaMalloc(&c->arena, k.total) != cudaSuccess) {
        c->arena = nullptr;
        cudaGetLastError();
        return CVC_ERR_NOMEM;
    }
    k.assign(static_cast<char*>(c->arena));
    for (int r = 0; r < Core::CORE_RING; r++) {
        if (cudaMallocHost((void**)&c->ring_sc[r], sizeof(SCall) * c->n) != cudaSuccess ||
            cudaMallocHost((void**)&c->ring_rs[r], sizeof(SResult) * c->n) != cudaSuccess) {
            cudaGetLastError();
            return CVC_ERR_NOMEM;
        }
        memset(c->ring_sc[r], 0, sizeof(SCall) * c->n);
        memset(c->ring_rs[r], 0, sizeof(SResult) * c->n);
        if (cudaEventCreateWithFlags(&c->ring_ev[r], cudaEventDisableTiming) != cudaSuccess) {
            c->ring_ev[r] = nullptr;
            cudaGetLastError();
            return CVC_ERR_CUDA;
        }
    }
    c->ring_slot = 0;
    c->h_sc = c->ring_sc[0];
    c->h_rs = c->ring_rs[0];
    bool ok = put(c->d_sd, c->sd) && put(c->d_pd, c->h_pd) && put(c->d_blk_colour, c->h_blk_colour) &&
              put(c->d_blk_plane, c->h_blk_plane) &&
              put(c->d_row_off, c->h_row_off) && put(c->d_row_w, c->h_row_w) &&
              put(c->d_row_stream, c->h_row_stream) && put(c->d_row_low, c->h_row_low) &&
              put(c->d_comp_tile0, c->h_comp_tile0) && put(c->d_tile_off, c->h_tile_off) &&
              put(c->d_tile_n, c->h_tile_n) && put(c->d_tile_w, c->h_tile_w) && put(c->d_tile_stream, c->h_tile_stream) &&
              put(c->d_tile_low, c->h_tile_low) && put(c->d_comp_stream, c->h_comp_stream) &&
              put(c->d_comp_low, c->h_comp_low) && put(c->d_comp_elem, c->h_comp_elem) &&
              put(c->d_comp_level, c->h_comp_level) && put(c->d_comp_plane, c->h_comp_plane) &&
              put(c->d_row_comp, c->h_row_comp) && put(c->d_row_mc, c->h_row_mc) && put(c->d_comp_ey, c->h_comp_ey) &&
              put(c->d_comp_ex, c->h_comp_ex) && put(c->d_blk_motion, c->h_blk_motion);
    for (const auto& sp : c->scale) ok = ok && put(sp->d_desc, sp->h_desc) && put(sp->d_blk, sp->h_blk);
    // state buffers start at zero (no frame may read them before a K-frame)
    for (int b = 0; b < 2 && ok; b++)
        ok = cudaMemset(c->d_est_buf[b], 0, (size_t)c->ncoef * 2) == cudaSuccess &&
             cudaMemset(c->d_dst_buf[b], 0, (size_t)c->ncoef * 2) == cudaSuccess;
    // coder state: frame 0 next, the decoder waiting for a K-frame
    std::vector<SCtl> ctl(c->n);
    for (SCtl& t : ctl) {
        memset(&t, 0, sizeof(t));
        t.dec_next = -1;
    }
    ok = ok && put(c->d_ctl, ctl);
    ok = ok && cudaStreamCreateWithFlags(&c->cap_stream, cudaStreamNonBlocking) == cudaSuccess;
    ok = ok && cudaStreamCreateWithFlags(&c->side, cudaStreamNonBlocking) == cudaSuccess;
    for (int k = 0; k < 2 && ok; k++)
        ok = cudaEventCreateWithFlags(&c->ev_fork[k], cudaEventDisableTiming) == cudaSuccess &&
             cudaEventCreateWithFlags(&c->ev_join[k], cudaEventDisableTiming) == cudaSuccess;
    if (!ok) {
        cudaGetLastError();
        return CVC_ERR_CUDA;
    }
    c->pend_reset.assign(c->n, 0);
    return CVC_OK;
}

void core_reset(Core* c, int s) {
    for (int i = 0; i < c->n; i++)
        if (s < 0 || s == i) c->pend_reset[i] = 1;
}

bool core_begin(Core* c) {
    const int r = (c->ring_slot + 1) % Core::CORE_RING;
    if (c->ring_used[r] && cudaEventSynchronize(c->ring_ev[r]) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    c->ring_slot = r;
    c->h_sc = c->ring_sc[r];
    c->h_rs = c->ring_rs[r];
    memset(c->h_sc, 0, sizeof(SCall) * c->n);
    return true;
}

void core_drop_graphs(Core* c) {
    for (auto& sp : c->scale)
        for (int m = 0; m < 4; m++) {
            if (sp->gexec[m]) cudaGraphExecDestroy(sp->gexec[m]);
            sp->gexec[m] = nullptr;
            sp->gkernels[m] = 0;
        }
}

cvc_status core_set_fusion(Core* c, int levels) {
    if (levels < 0 || levels > CVC_MAX_LEVELS) return CVC_ERR_INVALID_ARG;
    // the old tables go: nothing may still be running on them
    if (cudaDeviceSynchronize() != cudaSuccess) {
        cudaGetLastError();
        return CVC_ERR_CUDA;
    }
    core_drop_graphs(c);
    auto rebuild = [&](CtEngine& e) {
        e.tail_levels = levels;
        const std::vector<PlaneRef> planes = e.planes;
        return engine_build(&e, planes, true);
    };
    bool ok = rebuild(c->eng);
    for (size_t sc = 1; sc < c->scale.size() && ok; sc++) ok = rebuild(c->scale[sc]->eng);
    if (!ok) {
        cudaGetLastError();
        return CVC_ERR_NOMEM;
    }
    return CVC_OK;
}

cvc_status core_set_dfb_threads(Core* c, int threads) {
    if (threads != 0 && threads != DFBB_THREADS && threads != DFBB_THREADS_WIDE) return CVC_ERR_INVALID_ARG;
    // captured graphs hold the old launches: nothing may still be running on them
    if (cudaDeviceSynchronize() != cudaSuccess) {
        cudaGetLastError();
        return CVC_ERR_CUDA;
    }
    core_drop_graphs(c);
    c->eng.dfbb_threads = threads;
    for (size_t sc = 1; sc < c->scale.size(); sc++) c->scale[sc]->eng.dfbb_threads = threads;
    return CVC_OK;
}

void core_scaled_size(const Core* c, int s, int scale, int* h, int* w) {
    const ColourGeom& g = c->sd[s].cg;
    const int f = 1 << scale;
    *h = (g.H + f - 1) >> scale;
    *w = (g.W + f - 1) >> scale;
}

namespace {

struct StageClock {
    Core* c;
    cudaStream_t st;
    bool on;
    void begin(int s) {
        if (on) cudaEventRecord(c->ev[s][0], st);
    }
    void end(int s, long long launches) {
        if (!on) return;
        cudaEventRecord(c->ev[s][1], st);
        c->ev_used[s] = true;
        c->t_launches[s] += launches;
    }
};

#define CK(x)                                   \
    do {                                        \
        cudaError_t e_ = (x);                   \
        if (e_ != cudaSuccess) return e_;       \
    } while (0)

// the launch sequence of one step; *nl = kernels launched
cudaError_t enqueue_direct(Core* c, int mode, int scale, cudaStream_t st, bool timed, long long* nl) {
    StageClock clk{c, st, timed};
    const int n = c->n;
    long long k = 0;
    *nl = 0;
    CK(cudaMemsetAsync(c->d_rs, 0, sizeof(SResult) * n, st));
    // the call records' coder-state fields from the device-resident state
    k_step_begin<<<(int)cdiv(n, 128), 128, 0, st>>>(c->d_sd, c->d_sc, c->d_ctl, n);
    CK(cudaGetLastError());
    k += 1;
    const RowTable rt{c->d_row_off, c->d_row_w, c->d_row_low, c->d_row_stream, c->d_row_comp, c->d_row_mc, c->nrows};
    const RleTiles tt{c->d_tile_off, c->d_tile_n, c->d_tile_w, c->d_tile_stream, c->d_tile_low, c->ntiles};
    const CompTable ct{c->d_comp_tile0, c->d_comp_low, c->d_comp_stream, c->d_comp_elem,
                       c->d_comp_level, c->d_comp_plane, c->d_comp_ey, c->d_comp_ex, c->ncomp};
    const bool motion = !c->h_blk_motion.empty();
    const int rpb = c->shape.rle_rows;
    const int rgrid = (int)cdiv(c->nrows, rpb);
    if (mode & STEP_ENC) {
        Bases B;
        memset(&B, 0, sizeof(B));
        B.p[B_IN] = c->d_planes;
        B.p[B_COEF] = c->d_coef;
        B.p[B_WORK] = c->d_work;
        // the transform skips the planes of streams that do not encode in this call
        B.act = reinterpret_cast<const int*>(reinterpret_cast<const char*>(c->d_sc) + offsetof(SCall, enc_on));
        B.act_stride = (int)sizeof(SCall);
        // S1-S3: colour, 4:2:0, padding
        clk.begin(0);
        k_colour_fwd_b<<<(int)c->h_blk_colour.size(), 256, 0, st>>>(c->d_sd, c->d_sc, c->d_blk_colour, c->d_planes,
                                                                    c->d_luma[0], c->d_luma[1]);
        CK(cudaGetLastError());
        clk.end(0, 1);
        // S4, S5: LP analysis, DFB analysis
        clk.begin(1);
        CK(engine_run_part(&c->eng, FWD, 0, B, st));
        clk.end(1, engine_part_launches(&c->eng, FWD, 0));
        // the pyramid tails (coarse levels) on the side stream, beside the DFB stages of the others
        const int ntail = engine_part_launches(&c->eng, FWD, 2);
        if (ntail) {
            CK(cudaEventRecord(c->ev_fork[0], st));
            CK(cudaStreamWaitEvent(c->side, c->ev_fork[0], 0));
            CK(engine_run_part(&c->eng, FWD, 2, B, c->side));
            CK(cudaEventRecord(c->ev_join[0], c->side));
        }
        clk.begin(2);
        CK(engine_run_part(&c->eng, FWD, 1, B, st));
        if (ntail) CK(cudaStreamWaitEvent(st, c->ev_join[0], 0));
        clk.end(2, engine_part_launches(&c->eng, FWD, 1) + ntail);
        k += 1 + engine_part_launches(&c->eng, FWD, 0) + engine_part_launches(&c->eng, FWD, 1) + ntail;
        // S6-S8: normalise, threshold, quantise, K/P differencing
        clk.begin(3);
        launch_quant_b(c->quant_pow2, (int)c->h_blk_plane.size(), st, c->d_coef, c->d_est_buf[0], c->d_est_buf[1],
                       c->d_pd, c->d_blk_plane, c->d_sd, c->d_sc, c->d_res, c->d_rs);
        CK(cudaGetLastError());
        if (motion) {
            // §3.2 motion search, then the residuals of the motion-compensated P-frames
            k_motion_b<<<(int)c->h_blk_motion.size(), c->motion_threads, c->motion_smem, st>>>(
                c->d_sd, c->d_sc, c->d_blk_motion, c->d_luma[0], c->d_luma[1], c->d_mv, c->motion_ws);
            k_mc_resid_b<<<rgrid, 32 * rpb, 0, st>>>(c->d_est_buf[0], c->d_est_buf[1], rt, ct, c->d_sd, c->d_sc,
                                                     c->d_mv, c->d_res);
            CK(cudaGetLastError());
            k += 2;
        }
        clk.end(3, motion ? 3 : 1);
        // S9: RLE rows, row offsets, tokens, headers
        clk.begin(4);
        k_rle_count_b<<<c->ntiles, RLE_THREADS, 0, st>>>(c->d_res, tt, c->d_sc, c->d_tilecnt);
        CK(cudaGetLastError());
        CK(exclusive_scan(c->d_tilecnt, (uint32_t)c->ntiles, c->d_tileoff, c->d_scan_tmp, st));
        k_rle_write_b<<<c->ntiles, RLE_THREADS, 0, st>>>(c->d_res, tt, c->d_sd, c->d_sc, c->d_tileoff, c->d_rs);
        k_stream_header_b<<<n, 256, 0, st>>>(c->d_sd, c->d_sc, c->d_tileoff, ct, c->d_mv, c->d_rs);
        CK(cudaGetLastError());
        clk.end(4, 6);
        k += 7;
    }
    if (mode & STEP_DEC) {
        const int tg = c->shape.tok_blocks;
        // parse, token -> element counts, positions, checks, scatter of non-zero codes
        clk.begin(5);
        k_dec_parse_b<<<n, 1024, 0, st>>>(c->d_sd, c->d_sc, c->d_rs, ct, c->d_comp_tok, c->d_rs);
        k_dec_base_b<<<1, 32, 0, st>>>(c->d_sd, n, c->d_rs, c->d_tok_base, c->d_dtile_base);
        k_dec_count_b<<<tg, DEC_THREADS, 0, st>>>(c->d_sd, c->d_sc, c->d_rs, c->d_dtile_base, n, c->d_comp_tok, ct,
                                                 c->d_dtile_sum, c->d_rs);
        CK(cudaGetLastError());
        CK(exclusive_scan_dev(c->d_dtile_sum, c->d_dtile_base + n, (uint32_t)c->max_dtiles, c->d_dtile_pre,
                              c->d_scan_tmp2, st));
        CK(cudaMemsetAsync(c->d_res, 0, (size_t)c->ncoef * 2, st));
        CK(cudaMemsetAsync(c->d_comp_codes, 0, (size_t)c->ncomp * 4, st));
        k_dec_scatter_b<<<tg, DEC_THREADS, 0, st>>>(c->d_sd, c->d_sc, c->d_rs, c->d_dtile_base, n, c->d_comp_tok, ct,
                                                   c->d_dtile_pre, c->d_comp_codes, c->d_res);
        k_dec_check_b<<<(int)cdiv(c->ncomp, 256), 256, 0, st>>>(c->d_sd, c->d_rs, c->d_comp_codes, ct, c->d_rs);
        CK(cudaGetLastError());
        clk.end(5, 8);
        // inverse K/P differencing and dequantisation
        clk.begin(6);
        k_unquant_b<<<(int)c->h_blk_plane.size(), ELEM_THREADS, 0, st>>>(
            c->d_res, c->d_dst_buf[0], c->d_dst_buf[1], c->d_pd, c->d_blk_plane, c->d_sd, c->d_sc, c->d_rs, c->d_dcoef);
        k_unquant_keylow_b<<<(int)cdiv(c->lowcols, 256), 256, 0, st>>>(c->d_res, c->d_dst_buf[0], c->d_dst_buf[1],
                                                                       c->d_pd, c->nplanes, c->d_sd, c->d_sc, c->d_rs,
                                                                       c->d_dcoef);
        CK(cudaGetLastError());
        if (motion) {
            k_mc_recon_b<<<rgrid, 32 * rpb, 0, st>>>(c->d_res, c->d_dst_buf[0], c->d_dst_buf[1], rt, ct, c->d_sd,
                                                     c->d_sc, c->d_rs, c->d_dcoef);
            CK(cudaGetLastError());
            k += 1;
        }
        clk.end(6, motion ? 3 : 2);
        // inverse transform of the scale: DFB synthesis, then LP synthesis
        const ScalePlan& sp = *c->scale[scale];
        const CtEngine* ie = scale == 0 ? &c->eng : &sp.eng;
        Bases B;
        memset(&B, 0, sizeof(B));
        B.p[B_COEF] = c->d_dcoef;
        B.p[B_WORK] = c->d_work;
        B.p[B_OUT] = c->d_rplanes;
        // ... and of those that do not decode
        B.act = reinterpret_cast<const int*>(reinterpret_cast<const char*>(c->d_sc) + offsetof(SCall, dec_on));
        B.act_stride = (int)sizeof(SCall);
        clk.begin(7);
        const int ntail = engine_part_launches(ie, INV, 2);
        if (ntail) {
            CK(cudaEventRecord(c->ev_fork[1], st));
            CK(cudaStreamWaitEvent(c->side, c->ev_fork[1], 0));
            CK(engine_run_part(ie, INV, 2, B, c->side));
            CK(cudaEventRecord(c->ev_join[1], c->side));
        }
        CK(engine_run_part(ie, INV, 1, B, st));
        if (ntail) CK(cudaStreamWaitEvent(st, c->ev_join[1], 0));
        clk.end(7, engine_part_launches(ie, INV, 1) + ntail);
        clk.begin(8);
        CK(engine_run_part(ie, INV, 0, B, st));
        clk.end(8, engine_part_launches(ie, INV, 0));
        // normalisation, rounding, chroma upsampling, inverse colour transform
        clk.begin(9);
        int ncol = 0;
        if (!sp.h_blk.empty()) {
            k_colour_inv_b<<<(int)sp.h_blk.size(), 256, 0, st>>>(sp.d_desc, c->d_sc, c->d_rs, sp.d_blk,
                                                                 c->d_rplanes, c->d_dcoef);
            CK(cudaGetLastError());
            ncol = 1;
        }
        clk.end(9, ncol);
        k += 8 + 2 + ncol + engine_part_launches(ie, INV, 1) + engine_part_launches(ie, INV, 0) + ntail;
    }
    // statuses, lengths and frame types; the coder state advances where the call succeeded
    k_step_commit<<<(int)cdiv(n, 128), 128, 0, st>>>(c->d_sd, c->d_sc, c->d_rs, c->d_ctl, n);
    CK(cudaGetLastError());
    k += 1;
    *nl = k;
    return cudaSuccess;
}

}  // namespace

cvc_status core_capture(Core* c, int mode, int scale) {
    if (mode < STEP_ENC || mode > STEP_ENCDEC || scale < 0 || scale > c->max_levels) return CVC_ERR_INVALID_ARG;
    if (mode == STEP_ENC) scale = 0;   // no decoder in the step
    ScalePlan& sp = *c->scale[scale];
    if (sp.gexec[mode]) return CVC_OK;
    if (cudaStreamBeginCapture(c->cap_stream, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
        cudaGetLastError();
        return CVC_ERR_CUDA;
    }
    long long nl = 0;
    cudaError_t e = enqueue_direct(c, mode, scale, c->cap_stream, false, &nl);
    cudaGraph_t g = nullptr;
    cudaError_t e2 = cudaStreamEndCapture(c->cap_stream, &g);
    if (e == cudaSuccess && e2 == cudaSuccess) e = cudaGraphInstantiate(&sp.gexec[mode], g, 0);
    if (g) cudaGraphDestroy(g);
    if (e != cudaSuccess || e2 != cudaSuccess) {
        sp.gexec[mode] = nullptr;
        cudaGetLastError();
        return CVC_ERR_CUDA;
    }
    sp.gkernels[mode] = nl;
    return CVC_OK;
}

cvc_status core_enqueue(Core* c, int mode, cudaStream_t st, int scale) {
    if (mode < STEP_ENC || mode > STEP_ENCDEC || scale < 0 || scale > c->max_levels) return CVC_ERR_INVALID_ARG;
    if (mode == STEP_ENC) scale = 0;
    // every decoder output buffer was checked for the scale the step writes
    for (int i = 0; i < c->n; i++)
        if (c->h_sc[i].dec_on && c->h_sc[i].dec_scale != scale) return CVC_ERR_INVALID_ARG;
    const bool graph = c->use_graphs && !c->timing;
    if (graph) {
        cvc_status s = core_capture(c, mode, scale);
        if (s != CVC_OK) return s;
    }
    // resets requested since the last step go with this one
    for (int i = 0; i < c->n; i++)
        if (c->pend_reset[i]) c->h_sc[i].reset = 1;
    // the records in, the step, the results out; the slot is free again once they are back
    const size_t n = (size_t)c->n;
    cudaError_t e = cudaMemcpyAsync(c->d_sc, c->h_sc, sizeof(SCall) * n, cudaMemcpyHostToDevice, st);
    long long nl = 0;
    if (e == cudaSuccess) {
        if (graph) {
            e = cudaGraphLaunch(c->scale[scale]->gexec[mode], st);
            nl = c->scale[scale]->gkernels[mode];
        } else {
            e = enqueue_direct(c, mode, scale, st, c->timing, &nl);
        }
    }
    if (e == cudaSuccess) e = cudaMemcpyAsync(c->h_rs, c->d_rs, sizeof(SResult) * n, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaEventRecord(c->ring_ev[c->ring_slot], st);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return CVC_ERR_CUDA;
    }
    c->ring_used[c->ring_slot] = true;
    for (int i = 0; i < c->n; i++) c->pend_reset[i] = 0;
    note_launches(nl);
    return CVC_OK;
}

void core_collect(Core* c) {
    for (int s = 0; s < CVC_NUM_STAGES; s++) {
        if (!c->ev_used[s]) continue;
        float ms = 0.f;
        if (cudaEventElapsedTime(&ms, c->ev[s][0], c->ev[s][1]) == cudaSuccess) c->t_ms[s] += ms;
        c->ev_used[s] = false;
    }
}

cvc_status core_set_timing(Core* c, bool on) {
    if (on) {
        for (int s = 0; s < CVC_NUM_STAGES; s++) {
            for (int e = 0; e < 2; e++)
                if (!c->ev[s][e] && cudaEventCreate(&c->ev[s][e]) != cudaSuccess) return CVC_ERR_CUDA;
            c->t_ms[s] = 0.0;
            c->t_launches[s] = 0;
            c->ev_used[s] = false;
        }
    }
    c->timing = on;
    return CVC_OK;
}

bool core_fill_call(Core* c, int s, int mode, const StreamIo& io, int scale) {
    const SDesc& D = c->sd[s];
    SCall& C = c->h_sc[s];
    memset(&C, 0, sizeof(C));
    const size_t row = (size_t)D.cg.W * 3;
    if ((mode & STEP_ENC) && io.rgb) {
        if (!io.out || io.pitch < row || ((uintptr_t)io.out & 3)) return false;
        C.enc_on = 1;
        C.rgb_in = io.rgb;
        C.pitch_in = (long long)io.pitch;
        C.out = io.out;
        C.out_cap = (long long)std::min<size_t>(io.out_cap, (size_t)1 << 62);
    }
    if ((mode & STEP_DEC) && io.rgb_out) {
        if (scale < 0 || scale > c->prm[s].levels) return false;
        int hs = 0, ws = 0;
        core_scaled_size(c, s, scale, &hs, &ws);
        if (io.pitch_out < (size_t)ws * 3) return false;
        C.dec_on = 1;
        C.rgb_out = io.rgb_out;
        C.pitch_out = (long long)io.pitch_out;
        if (mode == STEP_ENCDEC && C.enc_on) {
            C.in = C.out;   // the decoder reads this call's encoder output
            C.in_len = -1;
        } else {
            if (!io.in) return false;
            C.in = io.in;
            C.in_len = (long long)std::min<size_t>(io.in_len, (size_t)1 << 62);
        }
        C.dec_scale = scale;
    }
    return true;
}

int core_ring_slot(const Core* c) { return c->ring_slot; }

void core_commit(Core* c, int s, int mode, cvc_status* enc, cvc_status* dec, size_t* out_len, int* type,
                 int* dec_type, unsigned* dec_index) {
    (void)mode;
    core_commit_at(c, c->ring_slot, s, enc, dec, out_len, type, dec_type, dec_index);
}

void core_commit_at(Core* c, int ring_slot, int s, cvc_status* enc, cvc_status* dec, size_t* out_len, int* type,
                    int* dec_type, unsigned* dec_index) {
    const cvc_batch_result& R = c->ring_rs[ring_slot][s].res;
    if (enc) *enc = R.enc_status;
    if (dec) *dec = R.dec_status;
    if (out_len) *out_len = R.out_len;
    if (type) *type = R.frame_type;
    if (dec_type) *dec_type = R.dec_frame_type;
    if (dec_index) *dec_index = R.dec_frame_index;
}

cvc_status core_take_error(Core* c, int s, cudaStream_t st, cvc_status* err) {
    // the word is read and cleared in stream order: errors of calls queued before
    // this one on `st` are seen, later ones are kept for the next read
    int* word = &c->d_ctl[s].first_err;
    int v = 0;
    if (cudaMemcpyAsync(&v, word, sizeof(int), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaMemsetAsync(word, 0, sizeof(int), st) != cudaSuccess || cudaStreamSynchronize(st) != cudaSuccess) {
        cudaGetLastError();
        return CVC_ERR_CUDA;
    }
    *err = (cvc_status)v;
    return CVC_OK;
}

}  // namespace cvc
