// mm_api.cu -- the C ABI: context, device workspace and the call sequence.
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

}  // namespace

struct mm_ctx {
    mm_config cfg;
    cudaStream_t stream = nullptr;
    char err[512] = {0};
    // binning
    Buf bin_of, bin_count, bin_start, bin_cursor, sorted, scan_tmp;
    // clipping output
    Buf vol, cen, s_cnt, s_nb, s_sh, s_area, s_fc;
    // face compaction
    Buf emit_mask, conf_mask, partner, emit_cnt, conf_cnt, face_off, inc_off;
    Buf face_i, face_j, face_shift, face_area, face_normal, face_cen, inc_face;
    // hydro scratch
    Buf Wh, grad, flux, w_int, dt_int, tot_partial;
    DevStatus *st = nullptr;        // device
    DevStatus *st_host = nullptr;   // pinned
    int *cnt_host = nullptr;        // pinned: faces, incidences
    int64_t fcap = 0, icap = 0;
    int collect_stats = 1;
    MeshDev mesh{};
    bool have_mesh = false;
    Grid grid{};
    // per-stage timing (events recorded on the stream) and launch counting
    int timing = 0;
    std::vector<cudaEvent_t> events;
    std::vector<int> ev_stage;  // stage of each (begin, end) pair
    size_t ev_used = 0;
    int64_t launches = 0;
};

// Record the begin (or end) event of a stage when timing is on.
static void stage_mark(mm_ctx *c, int stage, bool begin)
{
    if (!c->timing) return;
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

// Grow a buffer to at least `bytes` (with headroom); contents are not kept.
static mm_status ensure(mm_ctx *c, Buf &b, size_t bytes)
{
    if (bytes == 0) bytes = 16;
    if (b.bytes >= bytes) return MM_OK;
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
    return h;
}

static mm_status check_cfg(mm_ctx *c, const mm_config *g)
{
    if (!g) return fail(c, MM_EINVAL, "config is NULL");
    if (!(g->gamma > 1.0) || !std::isfinite(g->gamma)) return fail(c, MM_EINVAL, "gamma must be > 1");
    if (!(g->cfl > 0.0)) return fail(c, MM_EINVAL, "cfl must be > 0");
    if (g->limiter < 0 || g->limiter > 2) return fail(c, MM_EINVAL, "limiter must be 0, 1 or 2");
    if (g->precision < 0 || g->precision > 1) return fail(c, MM_EINVAL, "precision must be 0 or 1");
    if (!(g->rho_floor > 0.0) || !(g->eps_floor >= 0.0)) return fail(c, MM_EINVAL, "floors must be positive");
    if (!(g->area_rel >= 0.0)) return fail(c, MM_EINVAL, "area_rel must be >= 0");
    return MM_OK;
}

static mm_status read_status(mm_ctx *c)
{
    const DevStatus &s = *c->st_host;
    if (s.flags == 0) return MM_OK;
    if (s.flags & ST_EINVAL)
        return fail(c, MM_EINVAL, "generator %d lies outside [0, box) or is not finite", s.bad_cell);
    if (s.flags & ST_EDEGEN)
        return fail(c, MM_EDEGENERATE, "cell %d: inconsistent cut (degenerate or coincident generators)",
                    s.bad_cell);
    return fail(c, MM_ECAPACITY,
                "cell %d exceeded a per-cell capacity (flags 0x%x: 2 candidates, 4 planes (%d), 8 vertices "
                "(%d), 16 vertices per cut (%d), 32 faces (%d), 64 search rings (%d))",
                s.bad_cell, s.flags, PMAX, TMAX, NSTAGE, MAXF, MAXRING);
}

static void fill_mesh(const mm_ctx *c, mm_mesh *out)
{
    const MeshDev &m = c->mesh;
    out->n = m.n;
    out->nfaces = m.nf;
    out->nincident = c->cnt_host[1];
    out->face_stride = m.fs;
    for (int d = 0; d < 3; ++d) out->box[d] = m.box[d];
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
    for (int d = 0; d < 3; ++d) m.box[d] = mm->box[d];
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
    return m;
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
    Buf *bufs[] = {&c->bin_of, &c->bin_count, &c->bin_start, &c->bin_cursor, &c->sorted, &c->scan_tmp,
                   &c->vol, &c->cen, &c->s_cnt, &c->s_nb, &c->s_sh, &c->s_area, &c->s_fc, &c->emit_mask,
                   &c->conf_mask, &c->partner, &c->emit_cnt, &c->conf_cnt, &c->face_off, &c->inc_off,
                   &c->face_i, &c->face_j, &c->face_shift, &c->face_area, &c->face_normal, &c->face_cen,
                   &c->inc_face, &c->Wh, &c->grad, &c->flux, &c->w_int, &c->dt_int, &c->tot_partial};
    for (Buf *b : bufs)
        if (b->p) cudaFree(b->p);
    for (cudaEvent_t e : c->events) cudaEventDestroy(e);
    if (c->st) cudaFree(c->st);
    if (c->st_host) cudaFreeHost(c->st_host);
    if (c->cnt_host) cudaFreeHost(c->cnt_host);
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
    if (n < 1 || n > MM_MAX_CELLS) return fail(c, MM_EINVAL, "n = %lld outside [1, %lld]", (long long)n, MM_MAX_CELLS);
    for (int d = 0; d < 3; ++d)
        if (!(box[d] > 0.0) || !std::isfinite(box[d])) return fail(c, MM_EINVAL, "box[%d] must be finite and > 0", d);
    cudaStream_t s = c->stream;

    // grid of bins about one generator wide
    Grid g{};
    const double spacing = std::cbrt(box[0] * box[1] * box[2] / (double)n);
    int64_t nbins = 1;
    for (int d = 0; d < 3; ++d) {
        int64_t gd = (int64_t)std::floor(box[d] / spacing);
        if (gd < 1) gd = 1;
        if (gd > 4096) gd = 4096;
        g.g[d] = (int)gd;
        g.bs[d] = box[d] / (double)gd;
        g.box[d] = box[d];
        nbins *= gd;
    }
    if (nbins > (int64_t)1 << 30) return fail(c, MM_EINVAL, "too many bins");
    c->grid = g;
    mm_status r;
    const int64_t ns = n * (int64_t)MAXF;
    const size_t scan_n = (size_t)((nbins > n ? nbins : n) + 1);
    if ((r = ensure(c, c->bin_of, n * sizeof(int))) || (r = ensure(c, c->bin_count, (nbins + 1) * sizeof(int))) ||
        (r = ensure(c, c->bin_start, (nbins + 1) * sizeof(int))) || (r = ensure(c, c->bin_cursor, nbins * sizeof(int))) ||
        (r = ensure(c, c->sorted, n * sizeof(double4_32a))) || (r = ensure(c, c->scan_tmp, scan_tmp_size(scan_n) * sizeof(int))) ||
        (r = ensure(c, c->vol, n * sizeof(double))) || (r = ensure(c, c->cen, 3 * n * sizeof(double))) ||
        (r = ensure(c, c->s_cnt, n * sizeof(int))) || (r = ensure(c, c->s_nb, ns * sizeof(int))) ||
        (r = ensure(c, c->s_sh, ns)) || (r = ensure(c, c->s_area, ns * sizeof(double))) ||
        (r = ensure(c, c->s_fc, 3 * ns * sizeof(double))) || (r = ensure(c, c->emit_mask, n * 8)) ||
        (r = ensure(c, c->conf_mask, n * 8)) || (r = ensure(c, c->partner, ns)) ||
        (r = ensure(c, c->emit_cnt, n * sizeof(int))) || (r = ensure(c, c->conf_cnt, n * sizeof(int))) ||
        (r = ensure(c, c->face_off, (n + 1) * sizeof(int))) || (r = ensure(c, c->inc_off, (n + 1) * sizeof(int))))
        return r;

    stage_mark(c, MM_STAGE_BIN, true);
    CK(cudaMemsetAsync(c->st, 0, sizeof(DevStatus), s));
    CK(cudaMemsetAsync(c->bin_count.p, 0, (nbins + 1) * sizeof(int), s));
    CK(cudaMemsetAsync(c->bin_cursor.p, 0, nbins * sizeof(int), s));
    launch_bin_count(pos, n, g, P<int>(c->bin_of), P<int>(c->bin_count), c->st, s);
    launch_scan(P<int>(c->bin_count), P<int>(c->bin_start), nbins, P<int>(c->scan_tmp), s);
    launch_bin_scatter(pos, n, P<int>(c->bin_of), P<int>(c->bin_start), P<int>(c->bin_cursor), P<double4_32a>(c->sorted), s);
    launch_bin_sort(P<int>(c->bin_start), nbins, P<double4_32a>(c->sorted), s);
    CKLAUNCH();
    stage_mark(c, MM_STAGE_BIN, false);
    c->launches += 6;

    Slots sl{P<int>(c->s_cnt), P<int>(c->s_nb), P<unsigned char>(c->s_sh), P<double>(c->s_area), P<double>(c->s_fc)};
    const double amin = c->cfg.area_rel * std::pow(box[0] * box[1] * box[2] / (double)n, 2.0 / 3.0);
    stage_mark(c, MM_STAGE_CLIP, true);
    launch_clip(P<double4_32a>(c->sorted), P<int>(c->bin_start), n, g, amin, c->cfg.precision, c->cfg.collect_stats,
                P<double>(c->vol),
                P<double>(c->cen), sl, c->st, s);
    CKLAUNCH();
    stage_mark(c, MM_STAGE_CLIP, false);
    c->launches += 1;
    stage_mark(c, MM_STAGE_FACES, true);
    launch_face_confirm(n, sl, P<unsigned long long>(c->emit_mask), P<unsigned long long>(c->conf_mask),
                        P<signed char>(c->partner), P<int>(c->emit_cnt), P<int>(c->conf_cnt), s);
    launch_scan(P<int>(c->emit_cnt), P<int>(c->face_off), n, P<int>(c->scan_tmp), s);
    launch_scan(P<int>(c->conf_cnt), P<int>(c->inc_off), n, P<int>(c->scan_tmp), s);
    CKLAUNCH();
    stage_mark(c, MM_STAGE_FACES, false);
    c->launches += 7;
    CK(cudaMemcpyAsync(c->st_host, c->st, sizeof(DevStatus), cudaMemcpyDeviceToHost, s));
    CK(cudaMemcpyAsync(&c->cnt_host[0], P<int>(c->face_off) + n, sizeof(int), cudaMemcpyDeviceToHost, s));
    CK(cudaMemcpyAsync(&c->cnt_host[1], P<int>(c->inc_off) + n, sizeof(int), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    if ((r = read_status(c))) return r;
    const int64_t nf = c->cnt_host[0], ni = c->cnt_host[1];
    if (nf > c->fcap) {
        const int64_t cap = nf + nf / 8 + 64;
        if ((r = ensure(c, c->face_i, cap * sizeof(int))) || (r = ensure(c, c->face_j, cap * sizeof(int))) ||
            (r = ensure(c, c->face_shift, cap * sizeof(int))) || (r = ensure(c, c->face_area, cap * sizeof(double))) ||
            (r = ensure(c, c->face_normal, 3 * cap * sizeof(double))) ||
            (r = ensure(c, c->face_cen, 3 * cap * sizeof(double))) || (r = ensure(c, c->flux, 5 * cap * sizeof(double))))
            return r;
        c->fcap = cap;
    }
    if (ni > c->icap) {
        const int64_t cap = ni + ni / 8 + 64;
        if ((r = ensure(c, c->inc_face, cap * sizeof(int)))) return r;
        c->icap = cap;
    }
    stage_mark(c, MM_STAGE_FACES, true);
    launch_face_write(n, pos, g, sl, P<unsigned long long>(c->emit_mask), P<unsigned long long>(c->conf_mask),
                      P<signed char>(c->partner), P<int>(c->face_off), P<int>(c->inc_off), P<int>(c->face_i),
                      P<int>(c->face_j), P<int>(c->face_shift), P<double>(c->face_area), P<double>(c->face_normal),
                      P<double>(c->face_cen), c->fcap, P<int>(c->inc_face), s);
    CKLAUNCH();
    stage_mark(c, MM_STAGE_FACES, false);
    c->launches += 1;

    MeshDev &m = c->mesh;
    m.n = n;
    m.nf = nf;
    m.fs = c->fcap;
    for (int d = 0; d < 3; ++d) m.box[d] = box[d];
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
    c->have_mesh = true;
    if (out) fill_mesh(c, out);
    return MM_OK;
}

static mm_status check_mesh(mm_ctx *c, const mm_mesh *mesh)
{
    if (!mesh) return fail(c, MM_EINVAL, "mesh is NULL");
    if (mesh->n < 1 || !mesh->cell_volume || !mesh->inc_off) return fail(c, MM_EINVAL, "mesh is not initialised");
    return MM_OK;
}

mm_status mm_gradients(mm_ctx *c, const mm_mesh *mesh, const double *W, double *grad)
{
    if (!c) return MM_EINVAL;
    mm_status r;
    if ((r = check_mesh(c, mesh))) return r;
    if (!W || !grad) return fail(c, MM_EINVAL, "null pointer argument");
    MeshDev m = mesh_from(mesh);
    launch_gradient(m, hydro_cfg(c->cfg), W, false, grad, nullptr, nullptr, c->stream);
    CKLAUNCH();
    c->launches += 1;
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
    launch_dt_init(dt, c->stream);
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
    HydroCfg h = hydro_cfg(c->cfg);
    if ((r = ensure(c, c->Wh, 5 * m.n * sizeof(double))) || (r = ensure(c, c->grad, 15 * m.n * sizeof(double))) ||
        (r = ensure(c, c->flux, 5 * (m.nf > 0 ? m.nf : 1) * sizeof(double))))
        return r;
    cudaStream_t s = c->stream;
    stage_mark(c, MM_STAGE_GRADIENT_HALF, true);
    launch_gradient(m, h, U, true, nullptr, P<double>(c->Wh), dt, s);
    stage_mark(c, MM_STAGE_GRADIENT_HALF, false);
    stage_mark(c, MM_STAGE_GRADIENT, true);
    launch_gradient(m, h, P<double>(c->Wh), false, P<double>(c->grad), nullptr, nullptr, s);
    stage_mark(c, MM_STAGE_GRADIENT, false);
    stage_mark(c, MM_STAGE_FACE_FLUX, true);
    launch_face_flux(m, h, pos, w, P<double>(c->Wh), P<double>(c->grad), P<double>(c->flux), s);
    stage_mark(c, MM_STAGE_FACE_FLUX, false);
    stage_mark(c, MM_STAGE_UPDATE, true);
    launch_update(m, h, P<double>(c->flux), dt, U, s);
    stage_mark(c, MM_STAGE_UPDATE, false);
    CKLAUNCH();
    c->launches += 4;
    return MM_OK;
}

mm_status mm_drift(mm_ctx *c, double *pos, int64_t n, const double *w, const double *dt, const double box[3])
{
    if (!c) return MM_EINVAL;
    if (!pos || !w || !dt || !box) return fail(c, MM_EINVAL, "null pointer argument");
    if (n < 1 || n > MM_MAX_CELLS) return fail(c, MM_EINVAL, "bad n");
    stage_mark(c, MM_STAGE_DRIFT, true);
    launch_drift(pos, n, w, dt, box, c->stream);
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
    mm_mesh mesh;
    if ((r = mm_tessellate(c, pos, n, box, &mesh))) return r;
    if ((r = ensure(c, c->w_int, 3 * n * sizeof(double))) || (r = ensure(c, c->dt_int, sizeof(double)))) return r;
    double *w = w_out ? w_out : P<double>(c->w_int);
    double *dt = dt_out ? dt_out : P<double>(c->dt_int);
    cudaStream_t s = c->stream;
    MeshDev m = c->mesh;
    HydroCfg h = hydro_cfg(c->cfg);
    stage_mark(c, MM_STAGE_MESH_VELOCITY, true);
    if (dt_fixed) {
        launch_mesh_velocity(m, h, pos, U, w, nullptr, s);
        CK(cudaMemcpyAsync(dt, dt_fixed, sizeof(double), cudaMemcpyDeviceToDevice, s));
        c->launches += 1;
    } else {
        launch_dt_init(dt, s);
        launch_mesh_velocity(m, h, pos, U, w, dt, s);
        c->launches += 2;
    }
    stage_mark(c, MM_STAGE_MESH_VELOCITY, false);
    CKLAUNCH();
    if ((r = mm_flux_step(c, &mesh, pos, w, dt, U))) return r;
    return mm_drift(c, pos, n, w, dt, box);
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
    return MM_OK;
}

}  // extern "C"
