// mm_api.cu -- the C ABI: context, device workspace and the call sequence.
//
// A mesh is a batch of B independent periodic boxes stored back to back; the
// single-box calls (mm_tessellate, mm_step, ...) use B = 1.  mm_tessellate
// waits once for the face count and sizes the face arrays exactly.
// mm_step_batched instead reserves fixed capacities, so the whole step has no
// host synchronisation and is captured once into a CUDA graph and replayed.
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <new>
#include <vector>

#include "mm_internal.cuh"

using namespace mm;

namespace {

struct Buf {
    void *p = nullptr;
    size_t bytes = 0;
};

// Identity of a captured batched step: replays are valid while all of it holds.
struct GraphKey {
    const void *pos = nullptr, *U = nullptr, *dt_out = nullptr;
    int64_t n = 0;
    int64_t tables_gen = 0;
    int nbox = 0;
    unsigned long long boxes_hash = 0;
    mm_config cfg{};
};

unsigned long long fnv1a(const void *data, size_t bytes, unsigned long long h)
{
    const unsigned char *p = static_cast<const unsigned char *>(data);
    for (size_t k = 0; k < bytes; ++k) {
        h ^= p[k];
        h *= 1099511628211ull;
    }
    return h;
}

}  // namespace

struct mm_ctx {
    mm_config cfg;
    cudaStream_t stream = nullptr;
    char err[512] = {0};
    // box tables
    Buf boxes_dev, boxL_dev, box_off_dev, cbox;
    BoxDev *boxes_host = nullptr;  // pinned staging
    double *boxL_host = nullptr;
    long long *box_off_host = nullptr;
    int nbox_cap = 0, nbox = 0;
    int64_t nbins = 0, tess_n = 0;
    int64_t tables_gen = 0;  // bumped whenever the box tables are rewritten
    // binning
    Buf bin_of, bin_count, bin_start, bin_cursor, sorted, sortedf, scan_tmp;
    // clipping output
    Buf vol, cen, s_cnt, s_nb, s_sh, s_area, s_fc;
    // cells re-clipped by the large clipper: the retry list and their overflow rows
    Buf retry, o_cnt, o_nb, o_sh, o_area, o_fc, o_emit, o_conf, o_partner;
    Buf cell_order;  // processing order of the incident-face kernels
    // mm_step_host: device copies of the host arrays, and the stream and
    // events that overlap their copies with the step
    Buf h_pos, h_U, h_dt;
    cudaStream_t copy_stream = nullptr;
    cudaEvent_t ev_start = nullptr, ev_u_in = nullptr, ev_u_done = nullptr, ev_u_out = nullptr;
    int64_t orows = 0;
    // face compaction
    Buf emit_mask, conf_mask, partner, emit_cnt, conf_cnt, face_off, inc_off;
    Buf face_i, face_j, face_shift, face_area, face_normal, face_cen, inc_face;
    // hydro scratch
    Buf Wh, grad, flux, w_int, dt_int, tot_partial, drift_box, drift_cbox;
    Buf fgeo, minv;  // per-face A n and d, per-cell M^-1 of the gradient
    Buf heun_U0;  // start-of-step charges of a Heun step
    // mixed-precision records
    Buf x_fij, x_fa, x_fq, x_ff, x_cw, x_ch, x_grad, x_wv, x_flux;
    DevStatus *st = nullptr;        // device
    DevStatus *st_host = nullptr;   // pinned
    int *cnt_host = nullptr;        // pinned: faces, incidences
    double *box3_host = nullptr;    // pinned: one box size for mm_drift
    int64_t fcap = 0, icap = 0;
    MeshDev mesh{};
    int64_t mesh_ninc = 0;
    bool have_mesh = false;
    // per-stage timing (events recorded on the stream) and launch counting
    int timing = 0;
    bool capturing = false;
    std::vector<cudaEvent_t> events;
    std::vector<int> ev_stage;  // stage of each (begin, end) pair
    size_t ev_used = 0;
    int64_t launches = 0;
    // captured batched step
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t gexec = nullptr;
    GraphKey gkey;
    int64_t graph_launches = 0;
};

// Record the begin (or end) event of a stage when timing is on.
static void stage_mark(mm_ctx *c, int stage, bool begin)
{
    if (!c->timing || c->capturing) return;
    if (c->ev_used == c->events.size()) {
        cudaEvent_t e;
        if (cudaEventCreate(&e) != cudaSuccess) return;
        c->events.push_back(e);
    }
    if (begin) {
        if (c->ev_used % 2 != 0) return;
        c->ev_stage.resize(c->ev_used / 2 + 1);
        c->ev_stage[c->ev_used / 2] = stage;
    } else if (c->ev_used % 2 != 1) {
        return;
    }
    cudaEventRecord(c->events[c->ev_used], c->stream);
    ++c->ev_used;
}

static mm_status fail(mm_ctx *c, mm_status s, const char *fmt, ...) __attribute__((format(printf, 3, 4)));
static mm_status fail(mm_ctx *c, mm_status s, const char *fmt, ...)
{
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(c->err, sizeof(c->err), fmt, ap);
    va_end(ap);
    return s;
}

#define CK(call)                                                                                         \
    do {                                                                                                 \
        cudaError_t e_ = (call);                                                                         \
        if (e_ != cudaSuccess)                                                                           \
            return fail(c, e_ == cudaErrorMemoryAllocation ? MM_ENOMEM : MM_ECUDA, "%s: %s (%s:%d)",     \
                        #call, cudaGetErrorString(e_), __FILE__, __LINE__);                              \
    } while (0)

#define CKLAUNCH()                                                                                       \
    do {                                                                                                 \
        cudaError_t e_ = cudaGetLastError();                                                             \
        if (e_ != cudaSuccess)                                                                           \
            return fail(c, MM_ECUDA, "kernel launch: %s (%s:%d)", cudaGetErrorString(e_), __FILE__,      \
                        __LINE__);                                                                       \
    } while (0)

static void stage_mark_cb(void *arg, int stage, bool begin) { stage_mark(static_cast<mm_ctx *>(arg), stage, begin); }

static void drop_graph(mm_ctx *c);

// Grow a buffer to at least `bytes` (with headroom); contents are not kept.
// A captured graph holds the old addresses, so growth discards it.
static mm_status ensure(mm_ctx *c, Buf &b, size_t bytes)
{
    if (bytes == 0) bytes = 16;
    if (b.bytes >= bytes) return MM_OK;
    if (c->capturing) return fail(c, MM_ECUDA, "workspace growth during stream capture");
    if (c->gexec) {
        CK(cudaStreamSynchronize(c->stream));
        drop_graph(c);
    }
    if (b.p) CK(cudaFree(b.p));
    b.p = nullptr;
    b.bytes = 0;
    size_t want = bytes + bytes / 8;
    CK(cudaMalloc(&b.p, want));
    b.bytes = want;
    return MM_OK;
}

template <class T>
static T *P(const Buf &b)
{
    return static_cast<T *>(b.p);
}

static HydroCfg hydro_cfg(const mm_config &g)
{
    HydroCfg h;
    h.gamma = g.gamma;
    h.cfl = g.cfl;
    h.eta = g.eta;
    h.chi = g.chi;
    h.zeta = g.zeta;
    h.theta = g.theta;
    h.rho_floor = g.rho_floor;
    h.eps_floor = g.eps_floor;
    h.limiter = g.limiter;
    h.regularize = g.regularize;
    h.riemann = g.riemann;
    h.entropy = g.entropy;
    h.mach_th = g.mach_th;
    h.igm1 = 1.0 / (g.gamma - 1.0);
    h.kmach = (g.gamma + 1.0) / (2.0 * g.gamma);
    h.rhoa_floor = g.rho_floor * (g.gamma - 1.0) * g.rho_floor * g.eps_floor / std::pow(g.rho_floor, g.gamma);
    return h;
}

static mm_status check_cfg(mm_ctx *c, const mm_config *g)
{
    if (!g) return fail(c, MM_EINVAL, "config is NULL");
    if (!(g->gamma > 1.0) || !std::isfinite(g->gamma)) return fail(c, MM_EINVAL, "gamma must be > 1");
    if (!(g->cfl > 0.0)) return fail(c, MM_EINVAL, "cfl must be > 0");
    if (g->limiter < 0 || g->limiter > 3) return fail(c, MM_EINVAL, "limiter must be 0, 1, 2 or 3");
    if (g->entropy != 0 && g->entropy != 1) return fail(c, MM_EINVAL, "entropy must be 0 or 1");
    if (g->entropy && g->precision != 0)
        return fail(c, MM_EINVAL, "the entropy column needs the FP64 hydro path (precision 0)");
    if (g->entropy && !(g->mach_th >= 0.0)) return fail(c, MM_EINVAL, "mach_th must be >= 0");
    if (g->integrator != 0 && g->integrator != 1) return fail(c, MM_EINVAL, "integrator must be 0 or 1");
    if (g->integrator == 1 && (g->precision != 0 || g->entropy))
        return fail(c, MM_EINVAL, "Heun integration needs FP64 hydro without the entropy column");
    if (g->riemann < 0 || g->riemann > 1) return fail(c, MM_EINVAL, "riemann must be 0 (HLLC) or 1 (HLL)");
    if (g->precision < 0 || g->precision > 1) return fail(c, MM_EINVAL, "precision must be 0 or 1");
    if (!(g->rho_floor > 0.0) || !(g->eps_floor >= 0.0)) return fail(c, MM_EINVAL, "floors must be positive");
    if (!(g->area_rel >= 0.0)) return fail(c, MM_EINVAL, "area_rel must be >= 0");
    if (g->clip_warps < 1 || g->clip_warps > CLIP_MAX_WARPS) return fail(c, MM_EINVAL, "clip_warps must be in [1, 8]");
    if (g->cand_cap < 32 || g->cand_cap > 64) return fail(c, MM_EINVAL, "cand_cap must be in [32, 64]");
    if (!(g->bin_scale >= 0.25 && g->bin_scale <= 4.0)) return fail(c, MM_EINVAL, "bin_scale must be in [0.25, 4]");
    if (g->clip_sort != 0 && g->clip_sort != 1) return fail(c, MM_EINVAL, "clip_sort must be 0 or 1");
    return MM_OK;
}

static mm_status read_status(mm_ctx *c)
{
    const DevStatus &s = *c->st_host;
    if (s.flags == 0) return MM_OK;
    if (s.flags & ST_EINVAL)
        return fail(c, MM_EINVAL, "generator %d lies outside [0, box) or is not finite", s.bad_cell);
    if (s.flags & ST_EDEGEN)
        return fail(c, MM_EDEGENERATE, "cell %d: two generators at one position", s.bad_cell);
    if (s.flags & ST_ECAP_MESH)
        return fail(c, MM_ECAPACITY, "the batch has more faces than its fixed capacity (%lld faces, %lld incidences)",
                    (long long)c->fcap, (long long)c->icap);
    if (s.flags & ST_ECAP_RETRY)
        return fail(c, MM_ECAPACITY,
                    "%d cells overflowed the main clipper's per-cell lists, more than the %lld overflow rows "
                    "reserved for a captured batch",
                    s.nretry, (long long)c->orows);
    // name every per-cell capacity that overflowed, with its limit (before the
    // mesh inconsistency: a cell left without faces by an overflow leaves its
    // neighbours' faces unconfirmed too)
    struct Cap {
        int bit;
        const char *what;
        int limit;
    };
    const Cap caps[] = {{ST_ECAP_CAND, "candidates per sorted batch", 64},
                        {ST_ECAP_PLANE, "clipping planes per cell", PMAX},
                        {ST_ECAP_TRI, "vertices per cell", TMAX},
                        {ST_ECAP_STAGE, "vertices created by one cut", NSTAGE},
                        {ST_ECAP_FACE, "faces written per cell", MAXF},
                        {ST_ECAP_RING, "neighbour search rings", MAXRING}};
    char list[320] = {0};
    // a cell reported here overflowed the large clipper too (planes 128,
    // vertices 256, faces 128), after the main one's capacities below
    size_t used = 0;
    for (const Cap &k : caps)
        if ((s.flags & k.bit) && used < sizeof(list))
            used += (size_t)snprintf(list + used, sizeof(list) - used, "%s%s (limit %d)", used ? ", " : "", k.what,
                                     k.limit);
    if (used || !(s.flags & ST_EDEGEN_CUT))
        return fail(c, MM_ECAPACITY, "cell %d exceeded a per-cell capacity: %s", s.bad_cell, used ? list : "unknown");
    return fail(c, MM_EDEGENERATE,
                "cell %d: inconsistent mesh (near-degenerate generators): a cut inconsistent under both tie rules, "
                "or a face its neighbour does not have", s.bad_cell);
}

static void fill_mesh(const mm_ctx *c, mm_mesh *out)
{
    const MeshDev &m = c->mesh;
    out->n = m.n;
    out->nfaces = m.nf;
    out->nincident = c->mesh_ninc;
    out->face_stride = m.fs;
    out->nboxes = c->nbox;
    for (int d = 0; d < 3; ++d) out->box[d] = c->boxL_host[d];
    out->cell_box = m.cbox;
    out->box_size = m.boxL;
    out->face_i = m.face_i;
    out->face_j = m.face_j;
    out->face_shift = m.face_shift;
    out->face_area = m.area;
    out->face_normal = m.normal;
    out->face_centroid = m.fcen;
    out->cell_volume = m.vol;
    out->cell_centroid = m.cen;
    out->inc_off = m.inc_off;
    out->inc_face = m.inc_face;
}

static MeshDev mesh_from(const mm_mesh *mm)
{
    MeshDev m{};
    m.n = mm->n;
    m.nf = mm->nfaces;
    m.fs = mm->face_stride;
    m.nf_dev = nullptr;
    m.cbox = mm->cell_box;
    m.boxL = mm->box_size;
    m.face_i = mm->face_i;
    m.face_j = mm->face_j;
    m.face_shift = mm->face_shift;
    m.area = mm->face_area;
    m.normal = mm->face_normal;
    m.fcen = mm->face_centroid;
    m.vol = mm->cell_volume;
    m.cen = mm->cell_centroid;
    m.inc_off = mm->inc_off;
    m.inc_face = mm->inc_face;
    m.order = nullptr;  // a caller's mesh: cells in index order
    return m;
}

// Per-box tables: bins about one generator wide, bin ranges, face thresholds;
// uploaded through pinned staging, plus the cell -> box map.
static mm_status setup_boxes(mm_ctx *c, int64_t n, const int64_t *box_off, const double *boxL, int B)
{
    if (B < 1) return fail(c, MM_EINVAL, "need at least one box");
    if (n < 1 || n > MM_MAX_CELLS) return fail(c, MM_EINVAL, "n = %lld outside [1, %lld]", (long long)n, MM_MAX_CELLS);
    if (box_off[0] != 0 || box_off[B] != n) return fail(c, MM_EINVAL, "box offsets must run from 0 to n");
    if (B > c->nbox_cap) {
        CK(cudaStreamSynchronize(c->stream));
        if (c->boxes_host) cudaFreeHost(c->boxes_host);
        if (c->boxL_host) cudaFreeHost(c->boxL_host);
        if (c->box_off_host) cudaFreeHost(c->box_off_host);
        c->boxes_host = nullptr;
        c->boxL_host = nullptr;
        c->box_off_host = nullptr;
        c->nbox_cap = 0;
        CK(cudaMallocHost(&c->boxes_host, sizeof(BoxDev) * B));
        CK(cudaMallocHost(&c->boxL_host, sizeof(double) * 3 * B));
        CK(cudaMallocHost(&c->box_off_host, sizeof(long long) * (B + 1)));
        c->nbox_cap = B;
    } else {
        CK(cudaStreamSynchronize(c->stream));  // the staging may still feed an earlier copy
    }
    int64_t nbins = 0;
    for (int b = 0; b < B; ++b) {
        const int64_t nb = box_off[b + 1] - box_off[b];
        if (nb < 1) return fail(c, MM_EINVAL, "box %d holds no generator", b);
        const double *L = boxL + 3 * b;
        for (int d = 0; d < 3; ++d)
            if (!(L[d] >= MM_MIN_BOX && L[d] <= MM_MAX_BOX))
                return fail(c, MM_EINVAL, "box %d size %g outside [%g, %g]", b, L[d], MM_MIN_BOX, MM_MAX_BOX);
        BoxDev &g = c->boxes_host[b];
        const double vcell = L[0] * L[1] * L[2] / (double)nb;
        const double spacing = std::cbrt(vcell) * c->cfg.bin_scale;
        int64_t nbb = 1;
        for (int d = 0; d < 3; ++d) {
            int64_t gd = (int64_t)std::floor(L[d] / spacing);
            if (gd < 1) gd = 1;
            if (gd > 4096) gd = 4096;
            g.g[d] = (int)gd;
            g.bs[d] = L[d] / (double)gd;
            g.ibs[d] = (double)gd / L[d];
            g.L[d] = L[d];
            g.Lf[d] = (float)g.L[d];
            g.bsf[d] = (float)g.bs[d];
            g.ibsf[d] = (float)g.ibs[d];
            c->boxL_host[3 * b + d] = L[d];
            nbb *= gd;
        }
        g.bin_off = (int)nbins;
        g.amin = c->cfg.area_rel * std::pow(vcell, 2.0 / 3.0);
        nbins += nbb;
        if (nbins > ((int64_t)1 << 30)) return fail(c, MM_EINVAL, "too many bins");
    }
    for (int b = 0; b <= B; ++b) c->box_off_host[b] = (long long)box_off[b];
    mm_status r;
    if ((r = ensure(c, c->boxes_dev, sizeof(BoxDev) * B)) || (r = ensure(c, c->boxL_dev, sizeof(double) * 3 * B)) ||
        (r = ensure(c, c->box_off_dev, sizeof(long long) * (B + 1))) || (r = ensure(c, c->cbox, sizeof(int) * n)))
        return r;
    cudaStream_t s = c->stream;
    CK(cudaMemcpyAsync(c->boxes_dev.p, c->boxes_host, sizeof(BoxDev) * B, cudaMemcpyHostToDevice, s));
    CK(cudaMemcpyAsync(c->boxL_dev.p, c->boxL_host, sizeof(double) * 3 * B, cudaMemcpyHostToDevice, s));
    CK(cudaMemcpyAsync(c->box_off_dev.p, c->box_off_host, sizeof(long long) * (B + 1), cudaMemcpyHostToDevice, s));
    if (B == 1) {
        CK(cudaMemsetAsync(c->cbox.p, 0, sizeof(int) * n, s));
    } else {
        launch_fill_cbox(P<long long>(c->box_off_dev), B, n, P<int>(c->cbox), s);
        CKLAUNCH();
        c->launches += 1;
    }
    c->nbox = B;
    c->nbins = nbins;
    c->tess_n = n;
    c->tables_gen++;
    return MM_OK;
}

// Face arrays at capacity: exact (with headroom) after a counted pass, or
// fixed upfront in graph mode.
static mm_status ensure_faces(mm_ctx *c, int64_t nf, int64_t ni)
{
    mm_status r;
    if (nf > c->fcap) {
        const int64_t cap = nf + nf / 8 + 64;
        if ((r = ensure(c, c->face_i, cap * sizeof(int))) || (r = ensure(c, c->face_j, cap * sizeof(int))) ||
            (r = ensure(c, c->face_shift, cap * sizeof(int))) || (r = ensure(c, c->face_area, cap * sizeof(double))) ||
            (r = ensure(c, c->face_normal, 3 * cap * sizeof(double))) ||
            (r = ensure(c, c->face_cen, 3 * cap * sizeof(double))))
            return r;
        c->fcap = cap;
    }
    if (ni > c->icap) {
        const int64_t cap = ni + ni / 8 + 64;
        if ((r = ensure(c, c->inc_face, cap * sizeof(int)))) return r;
        c->icap = cap;
    }
    return MM_OK;
}

// Overflow rows for `rows` cells re-clipped by the large clipper.
static mm_status ensure_overflow(mm_ctx *c, int64_t rows)
{
    mm_status r;
    const int64_t ns = rows * (int64_t)MAXF_BIG;
    if ((r = ensure(c, c->o_cnt, rows * sizeof(int))) || (r = ensure(c, c->o_nb, ns * sizeof(int))) ||
        (r = ensure(c, c->o_sh, ns)) || (r = ensure(c, c->o_area, ns * sizeof(double))) ||
        (r = ensure(c, c->o_fc, 3 * ns * sizeof(double))) || (r = ensure(c, c->o_emit, 2 * rows * 8)) ||
        (r = ensure(c, c->o_conf, 2 * rows * 8)) || (r = ensure(c, c->o_partner, ns)))
        return r;
    c->orows = rows;
    return MM_OK;
}

static mm_status ensure_tess_buffers(mm_ctx *c, int64_t n)
{
    mm_status r;
    const int64_t nbins = c->nbins;
    const int64_t ns = n * (int64_t)MAXF;
    const size_t scan_n = (size_t)((nbins > n ? nbins : n) + 1);
    if ((r = ensure(c, c->bin_of, n * sizeof(int))) || (r = ensure(c, c->bin_count, (nbins + 1) * sizeof(int))) ||
        (r = ensure(c, c->bin_start, (nbins + 1) * sizeof(int))) || (r = ensure(c, c->bin_cursor, nbins * sizeof(int))) ||
        (r = ensure(c, c->sorted, n * sizeof(double4_32a))) || (r = ensure(c, c->sortedf, n * sizeof(float4))) ||
        (r = ensure(c, c->scan_tmp, scan_tmp_size(scan_n) * sizeof(int))) || (r = ensure(c, c->vol, n * sizeof(double))) ||
        (r = ensure(c, c->cen, 3 * n * sizeof(double))) || (r = ensure(c, c->s_cnt, n * sizeof(int))) ||
        (r = ensure(c, c->s_nb, ns * sizeof(int))) || (r = ensure(c, c->s_sh, ns)) ||
        (r = ensure(c, c->s_area, ns * sizeof(double))) || (r = ensure(c, c->s_fc, 3 * ns * sizeof(double))) ||
        (r = ensure(c, c->emit_mask, n * 8)) || (r = ensure(c, c->conf_mask, n * 8)) || (r = ensure(c, c->partner, ns)) ||
        (r = ensure(c, c->emit_cnt, n * sizeof(int))) || (r = ensure(c, c->conf_cnt, n * sizeof(int))) ||
        (r = ensure(c, c->face_off, (n + 1) * sizeof(int))) || (r = ensure(c, c->inc_off, (n + 1) * sizeof(int))) ||
        (r = ensure(c, c->retry, n * sizeof(int))) || (r = ensure(c, c->cell_order, n * sizeof(int))))
        return r;
    if (c->orows < RETRY_ROWS_FIXED && (r = ensure_overflow(c, RETRY_ROWS_FIXED))) return r;
    return MM_OK;
}

// Enqueue the tessellation of the boxes set up last.  fixed: the face arrays
// already have their capacities and the face count stays on the device.
static mm_status tess_enqueue(mm_ctx *c, const double *pos, bool fixed)
{
    const int64_t n = c->tess_n, nbins = c->nbins;
    cudaStream_t s = c->stream;
    mm_status r;
    stage_mark(c, MM_STAGE_BIN, true);
    CK(cudaMemsetAsync(c->st, 0, sizeof(DevStatus), s));
    CK(cudaMemsetAsync(c->bin_count.p, 0, (nbins + 1) * sizeof(int), s));
    CK(cudaMemsetAsync(c->bin_cursor.p, 0, nbins * sizeof(int), s));
    const BoxDev *boxes = P<BoxDev>(c->boxes_dev);
    const int *cbox = P<int>(c->cbox);
    launch_bin_count(pos, n, boxes, cbox, P<int>(c->bin_of), P<int>(c->bin_count), c->st, s);
    launch_scan(P<int>(c->bin_count), P<int>(c->bin_start), nbins, P<int>(c->scan_tmp), s);
    launch_bin_scatter(pos, n, P<int>(c->bin_of), P<int>(c->bin_start), P<int>(c->bin_cursor), P<double4_32a>(c->sorted), s);
    launch_bin_sort(P<int>(c->bin_start), nbins, P<double4_32a>(c->sorted), P<float4>(c->sortedf), s);
    CKLAUNCH();
    stage_mark(c, MM_STAGE_BIN, false);
    c->launches += 6;

    auto slots = [c]() {
        return Slots{P<int>(c->s_cnt), P<int>(c->s_nb), P<unsigned char>(c->s_sh), P<double>(c->s_area),
                     P<double>(c->s_fc), c->orows, P<int>(c->o_cnt), P<int>(c->o_nb), P<unsigned char>(c->o_sh),
                     P<double>(c->o_area), P<double>(c->o_fc), P<int>(c->retry)};
    };
    auto ovf = [c]() {
        return OvfFaces{P<unsigned long long>(c->o_emit), P<unsigned long long>(c->o_conf),
                        P<signed char>(c->o_partner), &c->st->nretry};
    };
    Slots sl = slots();
    const int prec = c->cfg.clip_filter ? 1 : 0;
    stage_mark(c, MM_STAGE_CLIP, true);
    launch_clip(P<double4_32a>(c->sorted), P<float4>(c->sortedf), P<int>(c->bin_start), n, boxes, cbox, prec,
                c->cfg.collect_stats,
                c->cfg.clip_warps, c->cfg.cand_cap, c->cfg.clip_sort, P<double>(c->vol), P<double>(c->cen), sl, c->st,
                s);
    // cells over a capacity of the main clipper, again with the large one
    // (one warp per overflow row; nothing to do when no cell overflowed)
    launch_clip_big(P<double4_32a>(c->sorted), P<float4>(c->sortedf), P<int>(c->bin_start), n, boxes, cbox, prec,
                    c->cfg.collect_stats, c->cfg.cand_cap, P<double>(c->vol), P<double>(c->cen), sl, c->st, s);
    CKLAUNCH();
    stage_mark(c, MM_STAGE_CLIP, false);
    c->launches += 2;
    stage_mark(c, MM_STAGE_FACES, true);
    launch_face_confirm(n, sl, ovf(), boxes, cbox, c->st, P<unsigned long long>(c->emit_mask), P<unsigned long long>(c->conf_mask),
                        P<signed char>(c->partner), P<int>(c->emit_cnt), P<int>(c->conf_cnt), s);
    launch_scan(P<int>(c->emit_cnt), P<int>(c->face_off), n, P<int>(c->scan_tmp), s);
    launch_scan(P<int>(c->conf_cnt), P<int>(c->inc_off), n, P<int>(c->scan_tmp), s);
    CKLAUNCH();
    c->launches += 7;
    int64_t nf = 0, ni = 0;
    if (!fixed) {
        stage_mark(c, MM_STAGE_FACES, false);
        for (int attempt = 0;; ++attempt) {
            CK(cudaMemcpyAsync(c->st_host, c->st, sizeof(DevStatus), cudaMemcpyDeviceToHost, s));
            CK(cudaMemcpyAsync(&c->cnt_host[0], P<int>(c->face_off) + n, sizeof(int), cudaMemcpyDeviceToHost, s));
            CK(cudaMemcpyAsync(&c->cnt_host[1], P<int>(c->inc_off) + n, sizeof(int), cudaMemcpyDeviceToHost, s));
            CK(cudaStreamSynchronize(s));
            // more cells overflowed than there were overflow rows: grow them to
            // the count and re-clip the list (its first rows again, harmlessly).
            // The cells not re-clipped yet had no faces, so their neighbours'
            // faces went unconfirmed: ST_EDEGEN_CUT alongside is expected, and
            // the second pass, from cleared flags, decides it again.
            const int fl = c->st_host->flags;
            if (attempt > 0 || !(fl & ST_ECAP_RETRY) || (fl & ~(ST_ECAP_RETRY | ST_EDEGEN_CUT))) break;
            if ((r = ensure_overflow(c, c->st_host->nretry))) return r;
            sl = slots();
            CK(cudaMemsetAsync(&c->st->flags, 0, sizeof(int), s));
            launch_clip_big(P<double4_32a>(c->sorted), P<float4>(c->sortedf), P<int>(c->bin_start), n, boxes, cbox,
                            prec, c->cfg.collect_stats, c->cfg.cand_cap, P<double>(c->vol), P<double>(c->cen), sl,
                            c->st, s);
            launch_face_confirm(n, sl, ovf(), boxes, cbox, c->st, P<unsigned long long>(c->emit_mask),
                                P<unsigned long long>(c->conf_mask), P<signed char>(c->partner), P<int>(c->emit_cnt),
                                P<int>(c->conf_cnt), s);
            launch_scan(P<int>(c->emit_cnt), P<int>(c->face_off), n, P<int>(c->scan_tmp), s);
            launch_scan(P<int>(c->conf_cnt), P<int>(c->inc_off), n, P<int>(c->scan_tmp), s);
            CKLAUNCH();
            c->launches += 8;
        }
        if ((r = read_status(c))) return r;
        nf = c->cnt_host[0];
        ni = c->cnt_host[1];
        if ((r = ensure_faces(c, nf, ni))) return r;
        stage_mark(c, MM_STAGE_FACES, true);
    }
    // the order in which the incident-face kernels take the cells (by face count)
    launch_cell_order(n, P<int>(c->inc_off), P<int>(c->cell_order), s);
    launch_face_write(n, pos, boxes, cbox, sl, ovf(), P<unsigned long long>(c->emit_mask), P<unsigned long long>(c->conf_mask),
                      P<signed char>(c->partner), P<int>(c->face_off), P<int>(c->inc_off), P<int>(c->face_i),
                      P<int>(c->face_j), P<int>(c->face_shift), P<double>(c->face_area), P<double>(c->face_normal),
                      P<double>(c->face_cen), c->fcap, P<int>(c->inc_face), c->icap, P<double>(c->vol),
                      P<double>(c->cen), c->st, s);
    CKLAUNCH();
    stage_mark(c, MM_STAGE_FACES, false);
    c->launches += 2;

    MeshDev &m = c->mesh;
    m.n = n;
    m.nf = fixed ? 0 : nf;
    m.fs = c->fcap;
    m.nf_dev = fixed ? P<int>(c->face_off) + n : nullptr;
    m.cbox = cbox;
    m.boxL = P<double>(c->boxL_dev);
    m.face_i = P<int>(c->face_i);
    m.face_j = P<int>(c->face_j);
    m.face_shift = P<int>(c->face_shift);
    m.area = P<double>(c->face_area);
    m.normal = P<double>(c->face_normal);
    m.fcen = P<double>(c->face_cen);
    m.vol = P<double>(c->vol);
    m.cen = P<double>(c->cen);
    m.inc_off = P<int>(c->inc_off);
    m.inc_face = P<int>(c->inc_face);
    m.order = P<int>(c->cell_order);
    c->mesh_ninc = fixed ? 0 : ni;
    c->have_mesh = true;
    return MM_OK;
}

// Hydro workspace for a mesh with n cells and face capacity fs.
static mm_status ensure_hydro(mm_ctx *c, int64_t n, int64_t fs)
{
    mm_status r;
    const int64_t F = fs > 0 ? fs : 1;
    if (c->cfg.precision == 1) {
        if ((r = ensure(c, c->x_fij, F * sizeof(int2))) || (r = ensure(c, c->x_fa, F * sizeof(float4))) ||
            (r = ensure(c, c->x_fq, F * sizeof(float4))) || (r = ensure(c, c->x_ff, F * sizeof(float2))) ||
            (r = ensure(c, c->x_flux, 2 * F * sizeof(float4))) || (r = ensure(c, c->x_cw, 2 * n * sizeof(float4))) ||
            (r = ensure(c, c->x_ch, 2 * n * sizeof(float4))) || (r = ensure(c, c->x_grad, 4 * n * sizeof(float4))) ||
            (r = ensure(c, c->x_wv, n * sizeof(float4))))
            return r;
    } else {
        // with the entropy column: 6 state rows, and 8 flux rows (the entropy
        // flux, each face's shock Mach number and its swept-volume rate)
        const int64_t ng = c->cfg.entropy ? 6 : 5, nfr = c->cfg.entropy ? 8 : 5;
        if ((r = ensure(c, c->Wh, ng * n * sizeof(double))) || (r = ensure(c, c->grad, 3 * ng * n * sizeof(double))) ||
            (r = ensure(c, c->flux, nfr * F * sizeof(double))) || (r = ensure(c, c->fgeo, 8 * F * sizeof(double))) ||
            (r = ensure(c, c->minv, 9 * n * sizeof(double))))
            return r;
    }
    return MM_OK;
}

// The hydro stages on mesh m (workspace already ensured).
static mm_status hydro_enqueue(mm_ctx *c, const MeshDev &m, const double *pos, const double *w, const double *dt,
                               double *U)
{
    HydroCfg h = hydro_cfg(c->cfg);
    cudaStream_t s = c->stream;
    if (c->cfg.precision == 1) {
        Mixed x{P<int2>(c->x_fij), P<float4>(c->x_fa), P<float4>(c->x_fq), P<float2>(c->x_ff), P<float4>(c->x_cw),
                P<float4>(c->x_ch), P<float4>(c->x_grad), P<float4>(c->x_wv), P<float4>(c->x_flux)};
        launch_mixed_step(m, h, pos, w, dt, x, U, s, stage_mark_cb, c);
        CKLAUNCH();
        c->launches += 6;
        return MM_OK;
    }
    stage_mark(c, MM_STAGE_GRADIENT_HALF, true);
    // states W^n = U / V, once per cell, in the gradient buffer (the second
    // gradient pass overwrites them only after the first has read them)
    launch_states(m, h, U, P<double>(c->grad), s);
    launch_face_geom(m, P<double>(c->fgeo), s);
    launch_gradient(m, h, P<double>(c->grad), P<double>(c->fgeo), P<double>(c->minv), false, nullptr,
                    P<double>(c->Wh), dt, s);
    stage_mark(c, MM_STAGE_GRADIENT_HALF, false);
    stage_mark(c, MM_STAGE_GRADIENT, true);
    // same mesh: M^-1 from the first pass
    launch_gradient(m, h, P<double>(c->Wh), P<double>(c->fgeo), P<double>(c->minv), true, P<double>(c->grad),
                    nullptr, nullptr, s);
    stage_mark(c, MM_STAGE_GRADIENT, false);
    stage_mark(c, MM_STAGE_FACE_FLUX, true);
    launch_face_flux(m, h, pos, w, P<double>(c->Wh), P<double>(c->grad), P<double>(c->flux), s);
    stage_mark(c, MM_STAGE_FACE_FLUX, false);
    stage_mark(c, MM_STAGE_UPDATE, true);
    launch_update(m, h, P<double>(c->flux), dt, U, s);
    stage_mark(c, MM_STAGE_UPDATE, false);
    CKLAUNCH();
    c->launches += 6;
    return MM_OK;
}

// One forward-Euler stage of Heun's method on mesh m: states W = U / V, their
// limited gradient, face fluxes reconstructed in space only, and the update.
static mm_status heun_stage(mm_ctx *c, const MeshDev &m, const double *pos, const double *w, const double *dt,
                            double *U)
{
    HydroCfg h = hydro_cfg(c->cfg);
    cudaStream_t s = c->stream;
    stage_mark(c, MM_STAGE_GRADIENT_HALF, true);
    launch_states(m, h, U, P<double>(c->Wh), s);
    stage_mark(c, MM_STAGE_GRADIENT_HALF, false);
    stage_mark(c, MM_STAGE_GRADIENT, true);
    launch_face_geom(m, P<double>(c->fgeo), s);
    launch_gradient(m, h, P<double>(c->Wh), P<double>(c->fgeo), P<double>(c->minv), false, P<double>(c->grad),
                    nullptr, nullptr, s);
    stage_mark(c, MM_STAGE_GRADIENT, false);
    stage_mark(c, MM_STAGE_FACE_FLUX, true);
    launch_face_flux(m, h, pos, w, P<double>(c->Wh), P<double>(c->grad), P<double>(c->flux), s);
    stage_mark(c, MM_STAGE_FACE_FLUX, false);
    stage_mark(c, MM_STAGE_UPDATE, true);
    launch_update(m, h, P<double>(c->flux), dt, U, s);
    stage_mark(c, MM_STAGE_UPDATE, false);
    CKLAUNCH();
    c->launches += 5;
    return MM_OK;
}

// Mesh velocity + per-box CFL timestep (or a copy of the fixed dt), the flux
// step and the drift, on the mesh of the last tessellation.  With
// integrator 1 (Heun): stage 1 on the start mesh, drift, a second
// tessellation, stage 2 on the end mesh with the same generator velocities,
// and the average of the start and stage-2 charges.
// Where a host step sends the final charges: U_host (ubytes), copied on the
// copy stream while the generators drift (the event ev_u_out marks its end),
// or on the stream after the step when the integrator finishes with U later.
struct HostOut {
    double *U_host;
    size_t ubytes;
    bool on_copy_stream;
};

static mm_status step_rest(mm_ctx *c, double *pos, double *U, const double *dt_fixed, double *w, double *dt,
                           bool fixed, HostOut *ho = nullptr)
{
    const MeshDev m = c->mesh;
    HydroCfg h = hydro_cfg(c->cfg);
    cudaStream_t s = c->stream;
    mm_status r;
    stage_mark(c, MM_STAGE_MESH_VELOCITY, true);
    if (dt_fixed) {
        launch_mesh_velocity(m, h, pos, U, w, nullptr, s);
        CK(cudaMemcpyAsync(dt, dt_fixed, sizeof(double) * c->nbox, cudaMemcpyDeviceToDevice, s));
        c->launches += 1;
    } else {
        launch_dt_init(dt, c->nbox, s);
        launch_mesh_velocity(m, h, pos, U, w, dt, s);
        c->launches += 2;
    }
    stage_mark(c, MM_STAGE_MESH_VELOCITY, false);
    CKLAUNCH();
    if (c->cfg.integrator == 1) {
        const size_t ubytes = sizeof(double) * 5 * (size_t)m.n;
        if ((r = ensure(c, c->heun_U0, ubytes))) return r;
        CK(cudaMemcpyAsync(c->heun_U0.p, U, ubytes, cudaMemcpyDeviceToDevice, s));
        if ((r = heun_stage(c, m, pos, w, dt, U))) return r;
    } else if ((r = hydro_enqueue(c, m, pos, w, dt, U))) {
        return r;
    }
    if (ho && c->cfg.integrator != 1) {
        // U is final: bring it back while the generators drift
        CK(cudaEventRecord(c->ev_u_done, s));
        CK(cudaStreamWaitEvent(c->copy_stream, c->ev_u_done, 0));
        CK(cudaMemcpyAsync(ho->U_host, U, ho->ubytes, cudaMemcpyDeviceToHost, c->copy_stream));
        CK(cudaEventRecord(c->ev_u_out, c->copy_stream));
        ho->on_copy_stream = true;
    }
    stage_mark(c, MM_STAGE_DRIFT, true);
    launch_drift(pos, m.n, w, dt, m.cbox, m.boxL, s);
    stage_mark(c, MM_STAGE_DRIFT, false);
    CKLAUNCH();
    c->launches += 1;
    if (c->cfg.integrator == 1) {
        if ((r = tess_enqueue(c, pos, fixed))) return r;
        if (!fixed && (r = ensure_hydro(c, c->mesh.n, c->mesh.fs))) return r;
        const MeshDev m1 = c->mesh;
        if ((r = heun_stage(c, m1, pos, w, dt, U))) return r;
        launch_heun_average(m1, h, P<double>(c->heun_U0), U, s);
        CKLAUNCH();
        c->launches += 1;
        if (ho) CK(cudaMemcpyAsync(ho->U_host, U, ho->ubytes, cudaMemcpyDeviceToHost, s));
    }
    return MM_OK;
}

static void drop_graph(mm_ctx *c)
{
    if (c->gexec) cudaGraphExecDestroy(c->gexec);
    if (c->graph) cudaGraphDestroy(c->graph);
    c->gexec = nullptr;
    c->graph = nullptr;
}

extern "C" {

void mm_default_config(mm_config *g)
{
    if (!g) return;
    std::memset(g, 0, sizeof(*g));
    g->gamma = 5.0 / 3.0;
    g->cfl = 0.3;
    g->eta = 1.0;
    g->chi = 1.0;
    g->zeta = 0.25;
    g->theta = 0.49;
    g->rho_floor = 1e-10;
    g->eps_floor = 1e-10;
    g->area_rel = 1e-10;
    g->limiter = 1;
    g->regularize = 0;
    g->precision = 0;
    g->riemann = 0;
    g->clip_warps = 2;  // fastest measured on the 256^3 shear layer (2: 367, 4: 378, 8: 414 ms)
    g->cand_cap = 64;
    g->clip_filter = 1;
    g->bin_scale = 1.0;
    g->mach_th = 1.1;
    g->entropy = 0;
    g->integrator = 0;
    g->clip_sort = 0;
}

mm_status mm_create(mm_ctx **out, const mm_config *cfg, void *cuda_stream)
{
    if (!out) return MM_EINVAL;
    *out = nullptr;
    mm_ctx *c = new (std::nothrow) mm_ctx();
    if (!c) return MM_ENOMEM;
    mm_status s = check_cfg(c, cfg);
    if (s != MM_OK) {
        delete c;
        return s;
    }
    c->cfg = *cfg;
    c->stream = static_cast<cudaStream_t>(cuda_stream);
    cudaError_t e = cudaMalloc(&c->st, sizeof(DevStatus));
    if (e == cudaSuccess) e = cudaMallocHost(&c->st_host, sizeof(DevStatus));
    if (e == cudaSuccess) e = cudaMallocHost(&c->cnt_host, 2 * sizeof(int));
    if (e == cudaSuccess) e = cudaMallocHost(&c->box3_host, 3 * sizeof(double));
    if (e != cudaSuccess) {
        mm_destroy(c);
        return e == cudaErrorMemoryAllocation ? MM_ENOMEM : MM_ECUDA;
    }
    *out = c;
    return MM_OK;
}

void mm_destroy(mm_ctx *c)
{
    if (!c) return;
    cudaStreamSynchronize(c->stream);
    drop_graph(c);
    Buf *bufs[] = {&c->boxes_dev, &c->boxL_dev, &c->box_off_dev, &c->cbox, &c->bin_of, &c->bin_count, &c->bin_start,
                   &c->bin_cursor, &c->sorted, &c->sortedf, &c->scan_tmp, &c->vol, &c->cen, &c->s_cnt, &c->s_nb, &c->s_sh,
                   &c->s_area, &c->s_fc, &c->emit_mask, &c->conf_mask, &c->partner, &c->emit_cnt, &c->conf_cnt,
                   &c->face_off, &c->inc_off, &c->face_i, &c->face_j, &c->face_shift, &c->face_area,
                   &c->face_normal, &c->face_cen, &c->inc_face, &c->Wh, &c->grad, &c->flux, &c->w_int, &c->dt_int,
                   &c->retry, &c->o_cnt, &c->o_nb, &c->o_sh, &c->o_area, &c->o_fc, &c->o_emit, &c->o_conf,
                   &c->o_partner, &c->cell_order, &c->h_pos, &c->h_U, &c->h_dt,
                   &c->tot_partial, &c->drift_box, &c->drift_cbox, &c->x_fij, &c->x_fa, &c->x_fq, &c->x_ff,
                   &c->x_cw, &c->x_ch, &c->x_grad, &c->x_wv, &c->x_flux, &c->heun_U0, &c->fgeo, &c->minv};
    if (c->copy_stream) cudaStreamSynchronize(c->copy_stream);
    for (Buf *b : bufs)
        if (b->p) cudaFree(b->p);
    for (cudaEvent_t e : c->events) cudaEventDestroy(e);
    for (cudaEvent_t e : {c->ev_start, c->ev_u_in, c->ev_u_done, c->ev_u_out})
        if (e) cudaEventDestroy(e);
    if (c->copy_stream) cudaStreamDestroy(c->copy_stream);
    if (c->st) cudaFree(c->st);
    if (c->st_host) cudaFreeHost(c->st_host);
    if (c->cnt_host) cudaFreeHost(c->cnt_host);
    if (c->box3_host) cudaFreeHost(c->box3_host);
    if (c->boxes_host) cudaFreeHost(c->boxes_host);
    if (c->boxL_host) cudaFreeHost(c->boxL_host);
    if (c->box_off_host) cudaFreeHost(c->box_off_host);
    delete c;
}

const char *mm_last_error(const mm_ctx *c) { return c ? c->err : "null context"; }

mm_status mm_set_config(mm_ctx *c, const mm_config *cfg)
{
    if (!c) return MM_EINVAL;
    mm_status s = check_cfg(c, cfg);
    if (s == MM_OK) c->cfg = *cfg;
    return s;
}

mm_status mm_tessellate(mm_ctx *c, const double *pos, int64_t n, const double box[3], mm_mesh *out)
{
    if (!c) return MM_EINVAL;
    c->have_mesh = false;
    if (!pos || !box) return fail(c, MM_EINVAL, "null pointer argument");
    const int64_t off[2] = {0, n};
    mm_status r;
    if ((r = setup_boxes(c, n, off, box, 1)) || (r = ensure_tess_buffers(c, n)) || (r = tess_enqueue(c, pos, false)))
        return r;
    if (out) fill_mesh(c, out);
    return MM_OK;
}

static mm_status check_mesh(mm_ctx *c, const mm_mesh *mesh)
{
    if (!mesh) return fail(c, MM_EINVAL, "mesh is NULL");
    if (mesh->n < 1 || !mesh->cell_volume || !mesh->inc_off || !mesh->cell_box || !mesh->box_size || mesh->nboxes < 1)
        return fail(c, MM_EINVAL, "mesh is not initialised");
    return MM_OK;
}

mm_status mm_gradients(mm_ctx *c, const mm_mesh *mesh, const double *W, double *grad)
{
    if (!c) return MM_EINVAL;
    mm_status r;
    if ((r = check_mesh(c, mesh))) return r;
    if (!W || !grad) return fail(c, MM_EINVAL, "null pointer argument");
    MeshDev m = mesh_from(mesh);
    if ((r = ensure(c, c->fgeo, 8 * (m.fs > 0 ? m.fs : 1) * sizeof(double)))) return r;
    launch_face_geom(m, P<double>(c->fgeo), c->stream);
    launch_gradient(m, hydro_cfg(c->cfg), W, P<double>(c->fgeo), nullptr, false, grad, nullptr, nullptr, c->stream);
    CKLAUNCH();
    c->launches += 2;
    return MM_OK;
}

mm_status mm_mesh_velocity(mm_ctx *c, const mm_mesh *mesh, const double *pos, const double *U, double *w)
{
    if (!c) return MM_EINVAL;
    mm_status r;
    if ((r = check_mesh(c, mesh))) return r;
    if (!pos || !U || !w) return fail(c, MM_EINVAL, "null pointer argument");
    launch_mesh_velocity(mesh_from(mesh), hydro_cfg(c->cfg), pos, U, w, nullptr, c->stream);
    CKLAUNCH();
    c->launches += 1;
    return MM_OK;
}

mm_status mm_timestep(mm_ctx *c, const mm_mesh *mesh, const double *U, const double *w, double *dt)
{
    if (!c) return MM_EINVAL;
    mm_status r;
    if ((r = check_mesh(c, mesh))) return r;
    if (!U || !w || !dt) return fail(c, MM_EINVAL, "null pointer argument");
    // the timestep of Sec. 4.2 measures |v - w| against the given w
    launch_dt_init(dt, (int)mesh->nboxes, c->stream);
    launch_timestep(mesh_from(mesh), hydro_cfg(c->cfg), U, w, dt, c->stream);
    CKLAUNCH();
    c->launches += 2;
    return MM_OK;
}

mm_status mm_flux_step(mm_ctx *c, const mm_mesh *mesh, const double *pos, const double *w, const double *dt,
                       double *U)
{
    if (!c) return MM_EINVAL;
    mm_status r;
    if ((r = check_mesh(c, mesh))) return r;
    if (!pos || !w || !dt || !U) return fail(c, MM_EINVAL, "null pointer argument");
    MeshDev m = mesh_from(mesh);
    if ((r = ensure_hydro(c, m.n, m.fs))) return r;
    return hydro_enqueue(c, m, pos, w, dt, U);
}

mm_status mm_drift(mm_ctx *c, double *pos, int64_t n, const double *w, const double *dt, const double box[3])
{
    if (!c) return MM_EINVAL;
    if (!pos || !w || !dt || !box) return fail(c, MM_EINVAL, "null pointer argument");
    if (n < 1 || n > MM_MAX_CELLS) return fail(c, MM_EINVAL, "bad n");
    for (int d = 0; d < 3; ++d)
        if (!(box[d] > 0.0) || !std::isfinite(box[d])) return fail(c, MM_EINVAL, "box[%d] must be finite and > 0", d);
    mm_status r;
    // one box: its own size table and an all-zero cell -> box map
    if ((r = ensure(c, c->drift_box, 3 * sizeof(double))) || (r = ensure(c, c->drift_cbox, n * sizeof(int)))) return r;
    CK(cudaStreamSynchronize(c->stream));  // the pinned staging may still feed an earlier copy
    for (int d = 0; d < 3; ++d) c->box3_host[d] = box[d];
    CK(cudaMemcpyAsync(c->drift_box.p, c->box3_host, 3 * sizeof(double), cudaMemcpyHostToDevice, c->stream));
    CK(cudaMemsetAsync(c->drift_cbox.p, 0, n * sizeof(int), c->stream));
    stage_mark(c, MM_STAGE_DRIFT, true);
    launch_drift(pos, n, w, dt, P<int>(c->drift_cbox), P<double>(c->drift_box), c->stream);
    stage_mark(c, MM_STAGE_DRIFT, false);
    CKLAUNCH();
    c->launches += 1;
    return MM_OK;
}

mm_status mm_step(mm_ctx *c, double *pos, double *U, int64_t n, const double box[3], const double *dt_fixed,
                  double *dt_out, double *w_out)
{
    if (!c) return MM_EINVAL;
    if (!pos || !U) return fail(c, MM_EINVAL, "null pointer argument");
    mm_status r;
    if ((r = mm_tessellate(c, pos, n, box, nullptr))) return r;
    if ((r = ensure(c, c->w_int, 3 * n * sizeof(double))) || (r = ensure(c, c->dt_int, sizeof(double))) ||
        (r = ensure_hydro(c, n, c->mesh.fs)))
        return r;
    double *w = w_out ? w_out : P<double>(c->w_int);
    double *dt = dt_out ? dt_out : P<double>(c->dt_int);
    return step_rest(c, pos, U, dt_fixed, w, dt, false);
}

mm_status mm_step_host(mm_ctx *c, double *pos, double *U, int64_t n, const double box[3], double *dt_out)
{
    if (!c) return MM_EINVAL;
    if (!pos || !U) return fail(c, MM_EINVAL, "null pointer argument");
    if (n < 1 || n > MM_MAX_CELLS) return fail(c, MM_EINVAL, "n = %lld outside [1, %lld]", (long long)n, MM_MAX_CELLS);
    const size_t pbytes = 3 * (size_t)n * sizeof(double);
    const size_t ubytes = (c->cfg.entropy ? 6 : 5) * (size_t)n * sizeof(double);
    mm_status r;
    if ((r = ensure(c, c->h_pos, pbytes)) || (r = ensure(c, c->h_U, ubytes)) || (r = ensure(c, c->h_dt, sizeof(double))))
        return r;
    if (!c->copy_stream) {
        // all or nothing, so that a later call never meets half of them
        cudaStream_t cs = nullptr;
        cudaEvent_t ev[4] = {nullptr, nullptr, nullptr, nullptr};
        cudaError_t e = cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking);
        for (int k = 0; k < 4 && e == cudaSuccess; ++k) e = cudaEventCreateWithFlags(&ev[k], cudaEventDisableTiming);
        if (e != cudaSuccess) {
            for (cudaEvent_t x : ev)
                if (x) cudaEventDestroy(x);
            if (cs) cudaStreamDestroy(cs);
            return fail(c, MM_ECUDA, "copy stream: %s", cudaGetErrorString(e));
        }
        c->copy_stream = cs;
        c->ev_start = ev[0]; c->ev_u_in = ev[1]; c->ev_u_done = ev[2]; c->ev_u_out = ev[3];
    }
    cudaStream_t s = c->stream, s2 = c->copy_stream;
    double *pd = P<double>(c->h_pos), *Ud = P<double>(c->h_U), *dtd = P<double>(c->h_dt);
    // the copy stream follows the work already queued (it may still read Ud)
    CK(cudaEventRecord(c->ev_start, s));
    CK(cudaStreamWaitEvent(s2, c->ev_start, 0));
    CK(cudaMemcpyAsync(pd, pos, pbytes, cudaMemcpyHostToDevice, s));
    CK(cudaMemcpyAsync(Ud, U, ubytes, cudaMemcpyHostToDevice, s2));
    CK(cudaEventRecord(c->ev_u_in, s2));
    HostOut ho{U, ubytes, false};
    r = mm_tessellate(c, pd, n, box, nullptr);
    if (r == MM_OK) r = ensure(c, c->w_int, 3 * n * sizeof(double));
    if (r == MM_OK) r = ensure_hydro(c, n, c->mesh.fs);
    if (r == MM_OK) {
        // the charges are first read by the mesh velocity
        CK(cudaStreamWaitEvent(s, c->ev_u_in, 0));
        r = step_rest(c, pd, Ud, nullptr, P<double>(c->w_int), dtd, false, &ho);
    }
    if (r != MM_OK) {
        cudaStreamSynchronize(s2);  // the host arrays stay in use until their copies end
        cudaStreamSynchronize(s);
        return r;
    }
    CK(cudaMemcpyAsync(pos, pd, pbytes, cudaMemcpyDeviceToHost, s));
    if (dt_out) CK(cudaMemcpyAsync(dt_out, dtd, sizeof(double), cudaMemcpyDeviceToHost, s));
    if (ho.on_copy_stream) CK(cudaStreamWaitEvent(s, c->ev_u_out, 0));
    CK(cudaStreamSynchronize(s));
    return MM_OK;
}

mm_status mm_step_batched(mm_ctx *c, double *pos, double *U, int64_t n, const int64_t *box_off, const double *boxes,
                          int nbox, double *dt_out)
{
    if (!c) return MM_EINVAL;
    if (!pos || !U || !box_off || !boxes) return fail(c, MM_EINVAL, "null pointer argument");
    if (!c->stream)
        return fail(c, MM_EINVAL, "a batched step is captured into a CUDA graph: give the context a non-default stream");
    if (nbox < 1) return fail(c, MM_EINVAL, "need at least one box");
    GraphKey key;
    key.pos = pos;
    key.U = U;
    key.dt_out = dt_out;
    key.n = n;
    key.nbox = nbox;
    key.boxes_hash = fnv1a(box_off, sizeof(int64_t) * (nbox + 1), 1469598103934665603ull);
    key.boxes_hash = fnv1a(boxes, sizeof(double) * 3 * nbox, key.boxes_hash);
    key.cfg = c->cfg;
    key.tables_gen = c->gkey.tables_gen;
    // the tables must still be the ones the graph was captured with
    const bool same = c->gexec && c->tables_gen == c->gkey.tables_gen && key.pos == c->gkey.pos &&
                      key.U == c->gkey.U && key.dt_out == c->gkey.dt_out &&
                      key.n == c->gkey.n && key.nbox == c->gkey.nbox && key.boxes_hash == c->gkey.boxes_hash &&
                      std::memcmp(&key.cfg, &c->gkey.cfg, sizeof(mm_config)) == 0;
    if (!same) {
        drop_graph(c);
        mm_status r;
        if ((r = setup_boxes(c, n, box_off, boxes, nbox)) || (r = ensure_tess_buffers(c, n))) return r;
        // fixed capacities: Voronoi cells of points in a box have < 8 unique faces on average
        const int64_t fcap = 10 * n + 1024, icap = 2 * fcap;
        if ((r = ensure_faces(c, fcap, icap)) || (r = ensure_hydro(c, n, c->fcap)) ||
            (r = ensure(c, c->w_int, 3 * n * sizeof(double))) || (r = ensure(c, c->dt_int, sizeof(double) * nbox)))
            return r;
        // nothing may be allocated while the stream is being captured
        if (c->cfg.integrator == 1 && (r = ensure(c, c->heun_U0, sizeof(double) * 5 * (size_t)n))) return r;
        CK(cudaStreamSynchronize(c->stream));
        const int64_t l0 = c->launches;
        c->capturing = true;
        cudaError_t e = cudaStreamBeginCapture(c->stream, cudaStreamCaptureModeThreadLocal);
        if (e != cudaSuccess) {
            c->capturing = false;
            return fail(c, MM_ECUDA, "cudaStreamBeginCapture: %s", cudaGetErrorString(e));
        }
        double *dt = P<double>(c->dt_int);
        r = tess_enqueue(c, pos, true);
        if (r == MM_OK) r = step_rest(c, pos, U, nullptr, P<double>(c->w_int), dt, true);
        if (r == MM_OK && dt_out) {
            e = cudaMemcpyAsync(dt_out, dt, sizeof(double) * nbox, cudaMemcpyDeviceToDevice, c->stream);
            if (e != cudaSuccess) r = fail(c, MM_ECUDA, "dt copy: %s", cudaGetErrorString(e));
        }
        cudaGraph_t g = nullptr;
        e = cudaStreamEndCapture(c->stream, &g);
        c->capturing = false;
        if (r != MM_OK) {
            if (g) cudaGraphDestroy(g);
            return r;
        }
        if (e != cudaSuccess) return fail(c, MM_ECUDA, "cudaStreamEndCapture: %s", cudaGetErrorString(e));
        c->graph = g;
        e = cudaGraphInstantiate(&c->gexec, g, 0);
        if (e != cudaSuccess) {
            drop_graph(c);
            return fail(c, MM_ECUDA, "cudaGraphInstantiate: %s", cudaGetErrorString(e));
        }
        c->gkey = key;
        c->gkey.tables_gen = c->tables_gen;
        c->graph_launches = c->launches - l0;
        c->launches = l0;
    }
    CK(cudaGraphLaunch(c->gexec, c->stream));
    c->launches += c->graph_launches;
    return MM_OK;
}

mm_status mm_get_config(const mm_ctx *c, mm_config *cfg)
{
    if (!c || !cfg) return MM_EINVAL;
    *cfg = c->cfg;
    return MM_OK;
}

mm_status mm_autotune(mm_ctx *c, const double *pos, int64_t n, const double box[3], int reps, double *best_ms)
{
    if (!c) return MM_EINVAL;
    if (!pos || !box) return fail(c, MM_EINVAL, "null pointer argument");
    if (reps < 1) reps = 1;
    static const int warps_opt[] = {2, 4, 8};
    static const int cap_opt[] = {32, 64};
    static const double scale_opt[] = {0.8, 1.0, 1.25, 1.5};
    static const int sort_opt[] = {0, 1};
    const mm_config keep = c->cfg;
    const int keep_timing = c->timing;
    cudaEvent_t e0, e1;
    CK(cudaEventCreate(&e0));
    CK(cudaEventCreate(&e1));
    double best = 1e300;
    mm_config best_cfg = keep;
    mm_status r = MM_OK;
    c->timing = 0;
    for (double sc : scale_opt)
        for (int wp : warps_opt)
            for (int cap : cap_opt)
                for (int so : sort_opt) {
                c->cfg = keep;
                c->cfg.bin_scale = sc;
                c->cfg.clip_warps = wp;
                c->cfg.cand_cap = cap;
                c->cfg.clip_sort = so;
                double tot = 0.0;
                for (int k = 0; k < reps + 1 && r == MM_OK; ++k) {
                    cudaEventRecord(e0, c->stream);
                    r = mm_tessellate(c, pos, n, box, nullptr);
                    cudaEventRecord(e1, c->stream);
                    cudaEventSynchronize(e1);
                    float ms = 0.0f;
                    cudaEventElapsedTime(&ms, e0, e1);
                    if (k > 0) tot += ms;  // the first run of each setting only warms up
                }
                if (r != MM_OK) break;
                if (tot / reps < best) {
                    best = tot / reps;
                    best_cfg = c->cfg;
                }
            }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    c->timing = keep_timing;
    c->cfg = keep;
    if (r != MM_OK) return r;
    c->cfg.bin_scale = best_cfg.bin_scale;
    c->cfg.clip_warps = best_cfg.clip_warps;
    c->cfg.cand_cap = best_cfg.cand_cap;
    c->cfg.clip_sort = best_cfg.clip_sort;
    if (best_ms) *best_ms = best;
    return MM_OK;
}

mm_status mm_sync_status(mm_ctx *c)
{
    if (!c) return MM_EINVAL;
    CK(cudaStreamSynchronize(c->stream));
    CK(cudaMemcpy(c->st_host, c->st, sizeof(DevStatus), cudaMemcpyDeviceToHost));
    return read_status(c);
}

mm_status mm_current_mesh(mm_ctx *c, mm_mesh *out)
{
    if (!c || !out) return MM_EINVAL;
    if (!c->have_mesh) return fail(c, MM_EINVAL, "no mesh yet");
    CK(cudaStreamSynchronize(c->stream));
    const int64_t n = c->mesh.n;
    CK(cudaMemcpy(&c->cnt_host[0], P<int>(c->face_off) + n, sizeof(int), cudaMemcpyDeviceToHost));
    CK(cudaMemcpy(&c->cnt_host[1], P<int>(c->inc_off) + n, sizeof(int), cudaMemcpyDeviceToHost));
    fill_mesh(c, out);
    out->nfaces = c->cnt_host[0];
    out->nincident = c->cnt_host[1];
    return MM_OK;
}

mm_status mm_prims_to_charges(mm_ctx *c, const mm_mesh *mesh, const double *rho, const double *vel,
                              const double *Pr, double *U)
{
    if (!c) return MM_EINVAL;
    mm_status r;
    if ((r = check_mesh(c, mesh))) return r;
    if (!rho || !vel || !Pr || !U) return fail(c, MM_EINVAL, "null pointer argument");
    launch_prims_to_charges(mesh_from(mesh), hydro_cfg(c->cfg), rho, vel, Pr, U, c->stream);
    CKLAUNCH();
    c->launches += 1;
    return MM_OK;
}

mm_status mm_totals(mm_ctx *c, const double *U, int64_t n, double *totals)
{
    if (!c) return MM_EINVAL;
    if (!U || !totals || n < 1) return fail(c, MM_EINVAL, "bad argument");
    const int nb = 256;
    mm_status r;
    if ((r = ensure(c, c->tot_partial, 2 * 5 * nb * sizeof(double)))) return r;
    launch_totals(U, n, P<double>(c->tot_partial), nb, totals, c->stream);
    CKLAUNCH();
    c->launches += 2;
    return MM_OK;
}

mm_status mm_copy(mm_ctx *c, void *dst, const void *src, int64_t bytes)
{
    if (!c) return MM_EINVAL;
    if (bytes < 0 || (bytes > 0 && (!dst || !src))) return fail(c, MM_EINVAL, "bad copy arguments");
    if (bytes == 0) return MM_OK;
    CK(cudaMemcpyAsync(dst, src, (size_t)bytes, cudaMemcpyDeviceToDevice, c->stream));
    return MM_OK;
}

mm_status mm_set_timing(mm_ctx *c, int on)
{
    if (!c) return MM_EINVAL;
    c->timing = on != 0;
    c->ev_used = 0;
    c->ev_stage.clear();
    return MM_OK;
}

mm_status mm_stage_times(mm_ctx *c, double ms[MM_NSTAGES], int64_t runs[MM_NSTAGES])
{
    if (!c || !ms || !runs) return MM_EINVAL;
    CK(cudaStreamSynchronize(c->stream));
    for (int k = 0; k < MM_NSTAGES; ++k) {
        ms[k] = 0.0;
        runs[k] = 0;
    }
    for (size_t p = 0; p + 1 < c->ev_used; p += 2) {
        float t = 0.0f;
        CK(cudaEventElapsedTime(&t, c->events[p], c->events[p + 1]));
        const int st = c->ev_stage[p / 2];
        ms[st] += t;
        runs[st] += 1;
    }
    return MM_OK;
}

int64_t mm_kernel_launches(const mm_ctx *c) { return c ? c->launches : 0; }

mm_status mm_tess_stats(mm_ctx *c, int64_t stats[MM_NSTATS])
{
    if (!c || !stats) return MM_EINVAL;
    CK(cudaMemcpyAsync(c->st_host, c->st, sizeof(DevStatus), cudaMemcpyDeviceToHost, c->stream));
    CK(cudaStreamSynchronize(c->stream));
    stats[0] = c->st_host->max_cand;
    stats[1] = c->st_host->max_planes;
    stats[2] = c->st_host->max_tris;
    stats[3] = c->st_host->multi_ring;
    stats[4] = (int64_t)c->st_host->cuts;
    stats[5] = (int64_t)c->st_host->pred64;
    stats[6] = (int64_t)c->st_host->solve64;
    stats[7] = (int64_t)c->st_host->fan64;
    stats[8] = (int64_t)c->st_host->tested;
    stats[9] = (int64_t)c->st_host->nretry;
    return MM_OK;
}

}  // extern "C"
