// fwi_api.cu -- the C ABI of libfwi (include/fwi.h): argument checks,
// workspace plan, and the order of kernels for each entry point.
//
// Order of one gradient (fwi_adjoint_gradient), after [Sec. 2] and [Sec. 3]:
//   c2 = (v dt/dx)^2 on the padded grid (+ velocity / stability checks)
//   forward time loop n = 0..nt-1 over all shots: u^{n+1}, traces d^n,
//     illumination, offset Hessian, sponge checkpoints        (fwi_step2d.cu)
//   residual r = d - d_obs and misfit; for Eq. 2 the adjoint source C^T C r
//   backward time loop m = nt-1..1: psi^m, u^{m-2}, imaging   (fwi_step2d.cu)
//   fold + 2/(v dx^2), illumination / offset-Hessian outputs, preconditioning
// Everything between the call's start and its final status read stays on the
// device and is queued on the caller's stream.
#include "fwi.h"
#include "fwi_internal.h"

#include <cudaTypedefs.h>

#include <nvtx3/nvToolsExt.h>

#include <algorithm>
#include <array>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <string>
#include <vector>

using namespace fwi;

namespace {

// NVTX range over one library call on the host timeline of a tracing tool
// (nsys and the like); without a tool attached the calls return at once.
struct Trace {
    explicit Trace(const char *name) { nvtxRangePushA(name); }
    ~Trace() { nvtxRangePop(); }
    Trace(const Trace &) = delete;
    Trace &operator=(const Trace &) = delete;
};

thread_local std::string t_err;
thread_local bool t_prof = false;
thread_local fwi_phase_times t_times{};
thread_local cudaEvent_t t_ev[4] = {nullptr, nullptr, nullptr, nullptr};
thread_local bool t_ev_recorded = false;
thread_local bool t_capturing = false; // recording a graph: events become graph nodes
thread_local int t_launch[3] = {0, 0, 0};

fwi_status fail(fwi_status s, const char *fmt, ...)
{
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    t_err = buf;
    return s;
}

fwi_status cuda_fail(cudaError_t e, const char *where)
{
    return fail(FWI_ERR_CUDA, "%s: %s", where, cudaGetErrorString(e));
}

// Stability limit of v dt / dx for the 8th-order / leapfrog pair in 2-D:
// (v dt/dx)^2 * 2 * max|symbol| <= 4, max|symbol| = 205/72 + 2(8/5 + 1/5 + 8/315 + 1/560).
constexpr float CFL_2D = FWI_CFL_LIMIT_2D;

constexpr size_t ALIGN = 256;
inline size_t align_up(size_t x, size_t a = ALIGN) { return (x + a - 1) / a * a; }

struct Part {
    size_t off = 0, bytes = 0;
};

struct Plan {
    Lay2D L{};
    int ns = 0, nt = 0, nrec = 0, hmax = -1, op = 0;
    bool with_offh = false; // forward kernel accumulates the offset Hessian
    bool need_bwd = false;  // adjoint pass (gradient / forward_save)
    bool need_seis_tab = false;
    bool born = false;      // Born modelling (u and du = J dv together)
    Tiling tf{}, tb{};
    Part scal, c2, damp, dc2, u[2], p[2], band, syn, acc_i, acc_h, acc_g, tab, sched;
    size_t tab_src = 0, tab_srcij = 0, tab_fptr = 0, tab_fent = 0, tab_bptr = 0, tab_bent = 0, tab_bshot = 0;
    Part adj_t; // adjoint source in backward-table order [nt][ns*nrec]
    Part prod;  // scale x receiver factor (fwi_precondition_receiver)
    Part dext;  // extended Born: planes D~(y, h), h = -HEXT_MAX..HEXT_MAX
    Part acc_ext; // extended migration: [2 HEXT_MAX + 1][nzp][nxp] image sums
    bool ext = false; // extended operators (64 x 8 tiles)
    // snapshot checkpoints (FWI_CKPT_SNAPSHOT): snapshot j holds level j*K
    bool snap = false;
    int snap_prec = FWI_SNAP_F32, K = 0, nck = 0;
    Tiling tr{};          // tiling of the segment re-propagation (plain forward)
    Part snaps, snap_max; // [nck][2][ns][fstride] F32 / 16-bit, [nck][2][ns]
    Part seg;             // segment levels beyond the two forward buffers
    size_t total = 0;
};

fwi_status check_grid(const fwi_grid *g)
{
    if (!g) return fail(FWI_ERR_INVALID_ARG, "grid is NULL");
    if (g->ndim != 2) return fail(FWI_ERR_INVALID_ARG, "ndim=%d: only 2-D grids are supported", g->ndim);
    if (g->ny != 1) return fail(FWI_ERR_INVALID_ARG, "ny must be 1 in 2-D (got %d)", g->ny);
    if (g->nz < 1 || g->nx < 1) return fail(FWI_ERR_INVALID_ARG, "nz=%d nx=%d must be >= 1", g->nz, g->nx);
    if (g->nt < 2) return fail(FWI_ERR_INVALID_ARG, "nt=%d must be >= 2", g->nt);
    if (g->sponge < 1 || g->sponge > 64) return fail(FWI_ERR_INVALID_ARG, "sponge=%d outside 1..64", g->sponge);
    if (!(g->dx > 0.f) || !std::isfinite(g->dx)) return fail(FWI_ERR_INVALID_ARG, "dx must be > 0");
    if (!(g->dt > 0.f) || !std::isfinite(g->dt)) return fail(FWI_ERR_INVALID_ARG, "dt must be > 0");
    if (!(g->vref > 0.f) || !std::isfinite(g->vref)) return fail(FWI_ERR_INVALID_ARG, "vref must be > 0");
    if (!(g->refl > 0.f && g->refl < 1.f)) return fail(FWI_ERR_INVALID_ARG, "refl must be in (0,1)");
    const long long nzp = g->nz + 2LL * g->sponge, nxp = g->nx + 2LL * g->sponge;
    if (nzp * (nxp + GXL + GXR + 32) >= (1LL << 31)) return fail(FWI_ERR_INVALID_ARG, "grid too large");
    return FWI_OK;
}

fwi_status check_geom(const fwi_grid *g, const fwi_geometry *ge, bool coords)
{
    if (!ge) return fail(FWI_ERR_INVALID_ARG, "geometry is NULL");
    if (ge->nshots < 1) return fail(FWI_ERR_INVALID_ARG, "nshots=%d must be >= 1", ge->nshots);
    if (ge->nrec < 0) return fail(FWI_ERR_INVALID_ARG, "nrec=%d must be >= 0", ge->nrec);
    if ((long long)ge->nshots * ge->nrec >= (1LL << 31)) return fail(FWI_ERR_INVALID_ARG, "too many receivers");
    if (!coords) return FWI_OK;
    if (!ge->src) return fail(FWI_ERR_INVALID_ARG, "geometry.src is NULL");
    if (ge->nrec > 0 && !ge->rec) return fail(FWI_ERR_INVALID_ARG, "geometry.rec is NULL");
    if (!ge->wavelet) return fail(FWI_ERR_INVALID_ARG, "geometry.wavelet is NULL");
    for (int s = 0; s < ge->nshots; ++s) {
        const int *c = ge->src + 3 * s;
        if (c[0] < 0 || c[0] >= g->nz || c[1] != 0 || c[2] < 0 || c[2] >= g->nx)
            return fail(FWI_ERR_INVALID_ARG, "source of shot %d at (%d,%d,%d) outside the model", s, c[0], c[1], c[2]);
        for (int r = 0; r < ge->nrec; ++r) {
            const int *q = ge->rec + 3 * ((long long)s * ge->nrec + r);
            if (q[0] < 0 || q[0] >= g->nz || q[1] != 0 || q[2] < 0 || q[2] >= g->nx)
                return fail(FWI_ERR_INVALID_ARG, "receiver %d of shot %d at (%d,%d,%d) outside the model", r, s, q[0], q[1], q[2]);
        }
    }
    return FWI_OK;
}

fwi_status check_opts(const fwi_options *o, int op)
{
    if (!o) {
        if (op == FWI_OP_FORWARD || op == FWI_OP_FORWARD_SAVE || op == FWI_OP_PRECONDITION || op == FWI_OP_BORN ||
            op == FWI_OP_GN_HVP || op == FWI_OP_MISFIT || op == FWI_OP_RECEIVER_FACTOR ||
            op == FWI_OP_PRECONDITION_RECEIVER || op == FWI_OP_EXT_BORN || op == FWI_OP_EXT_MIGRATION ||
            op == FWI_OP_PM_HESSIAN)
            return FWI_OK;
        return fail(FWI_ERR_INVALID_ARG, "options are NULL");
    }
    if (o->misfit != FWI_MISFIT_OLS && o->misfit != FWI_MISFIT_TIME_INTEGRAL)
        return fail(FWI_ERR_INVALID_ARG, "misfit=%d unknown", o->misfit);
    if (o->illum_mode != FWI_ILLUM_U2 && o->illum_mode != FWI_ILLUM_UTT2)
        return fail(FWI_ERR_INVALID_ARG, "illum_mode=%d unknown", o->illum_mode);
    if (o->hmax < -1 || o->hmax > FWI_HMAX_LIMIT)
        return fail(FWI_ERR_INVALID_ARG, "hmax=%d outside -1..%d", o->hmax, FWI_HMAX_LIMIT);
    if (o->precond < FWI_PRECOND_NONE || o->precond > FWI_PRECOND_OFFSET)
        return fail(FWI_ERR_INVALID_ARG, "precond=%d unknown", o->precond);
    if (o->precond == FWI_PRECOND_OFFSET && o->hmax < 0)
        return fail(FWI_ERR_INVALID_ARG, "precond=OFFSET needs hmax >= 0");
    if (!(o->eps > 0.f) || !std::isfinite(o->eps)) return fail(FWI_ERR_INVALID_ARG, "eps must be > 0");
    if (o->ckpt != FWI_CKPT_SPONGE && o->ckpt != FWI_CKPT_SNAPSHOT)
        return fail(FWI_ERR_INVALID_ARG, "ckpt=%d unknown", o->ckpt);
    if (o->snap_prec < FWI_SNAP_F32 || o->snap_prec > FWI_SNAP_F16S)
        return fail(FWI_ERR_INVALID_ARG, "snap_prec=%d unknown", o->snap_prec);
    if (o->snap_interval < 0) return fail(FWI_ERR_INVALID_ARG, "snap_interval=%d must be >= 0", o->snap_interval);
    if (o->shot_group < 0) return fail(FWI_ERR_INVALID_ARG, "shot_group=%d must be >= 0", o->shot_group);
    if (o->hess_v6 != 0 && o->hess_v6 != 1) return fail(FWI_ERR_INVALID_ARG, "hess_v6=%d must be 0 or 1", o->hess_v6);
    return FWI_OK;
}

Lay2D make_layout(const fwi_grid *g)
{
    Lay2D L{};
    L.nz = g->nz;
    L.nx = g->nx;
    L.P = g->sponge;
    L.nzp = g->nz + 2 * g->sponge;
    L.nxp = g->nx + 2 * g->sponge;
    L.pitch = (int)align_up((size_t)(GXL + L.nxp + GXR), 32);
    L.rows = L.nzp + 2 * GZ;
    L.fstride = (long long)align_up((size_t)L.rows * L.pitch, 64);
    L.nband = 2 * L.P * L.nxp + 2 * L.P * L.nz;
    L.nbandp = (L.nband + 3) / 4 * 4;
    L.dt = g->dt;
    L.dx = g->dx;
    const double etamax = 3.0 * g->vref * std::log(1.0 / g->refl) / (2.0 * g->sponge * g->dx);
    L.etamax_dt = (float)(etamax * g->dt);
    L.inv_p2 = (float)(1.0 / ((double)g->sponge * g->sponge));
    return L;
}

fwi_status make_plan(const fwi_grid *g, const fwi_geometry *ge, const fwi_options *o, int op,
                     bool coords, Plan &pl)
{
    fwi_status st;
    if ((st = check_grid(g)) != FWI_OK) return st;
    const bool no_geom = op == FWI_OP_PRECONDITION || op == FWI_OP_PRECONDITION_RECEIVER;
    if (!no_geom && (st = check_geom(g, ge, coords)) != FWI_OK) return st;
    if ((st = check_opts(o, op)) != FWI_OK) return st;
    pl.L = make_layout(g);
    pl.op = op;
    pl.nt = g->nt;
    const Lay2D &L = pl.L;
    size_t off = 0;
    auto take = [&](Part &p, size_t bytes) {
        p.off = off;
        p.bytes = bytes;
        off = align_up(off + bytes);
    };
    take(pl.scal, 256);
    const bool need_bwd = (op == FWI_OP_GRADIENT || op == FWI_OP_FORWARD_SAVE || op == FWI_OP_GN_HVP ||
                           op == FWI_OP_EXT_MIGRATION);
    const bool born = (op == FWI_OP_BORN || op == FWI_OP_GN_HVP || op == FWI_OP_EXT_BORN);
    pl.ext = (op == FWI_OP_EXT_BORN || op == FWI_OP_EXT_MIGRATION);
    if ((born || pl.ext) && o && o->ckpt != FWI_CKPT_SPONGE)
        return fail(FWI_ERR_INVALID_ARG, "Born modelling, Hessian-vector products and the extended operators use "
                                         "sponge checkpoints");
    pl.snap = need_bwd && o && o->ckpt == FWI_CKPT_SNAPSHOT;
    // scheduler counters: forward, backward, and (snapshots) re-propagation
    if (!no_geom) take(pl.sched, (size_t)(pl.snap ? 3 : 2) * g->nt * sizeof(int));
    if (no_geom) {
        if (op == FWI_OP_PRECONDITION_RECEIVER)
            take(pl.prod, (size_t)(FWI_HMAX_LIMIT + 1) * L.nz * L.nx * sizeof(float));
        pl.total = off;
        return FWI_OK;
    }
    pl.ns = ge->nshots;
    pl.nrec = ge->nrec;
    pl.hmax = o ? o->hmax : -1;
    pl.with_offh = (op == FWI_OP_GRADIENT || op == FWI_OP_OFFSET_HESSIAN) && pl.hmax >= 0;
    if (op == FWI_OP_OFFSET_HESSIAN && pl.hmax < 0)
        return fail(FWI_ERR_INVALID_ARG, "offset Hessian needs hmax >= 0");
    pl.need_bwd = need_bwd;
    pl.need_seis_tab = (op == FWI_OP_GRADIENT || op == FWI_OP_FORWARD || op == FWI_OP_FORWARD_SAVE ||
                        op == FWI_OP_MISFIT);
    pl.born = born;
    pl.tf = make_tiling(L, pl.ns, pl.with_offh ? STEP_FWD_OFFH : STEP_FWD, -1, 0, pl.hmax);
    // the Born step runs on the backward step's default 64 x 16 tiles, the
    // extended operators on its 64 x 8 tiles, in chunks of 32 shots (each
    // chunk loads the tile's 2 HE + 1 coefficient planes or flushes its
    // 2 HE + 1 image planes once)
    pl.tb = pl.ext ? make_tiling(L, pl.ns, STEP_BWD, 1, 32)
                   : (born ? make_tiling(L, pl.ns, STEP_BWD, 0) : make_tiling(L, pl.ns, STEP_BWD));
    const size_t fbytes = (size_t)L.fstride * sizeof(float);
    const size_t nphys = (size_t)L.nz * L.nx;
    take(pl.c2, fbytes);
    take(pl.damp, fbytes);
    if (op == FWI_OP_EXT_BORN) take(pl.dext, fbytes * (2 * HEXT_MAX + 1));
    if (op == FWI_OP_EXT_MIGRATION)
        take(pl.acc_ext, (size_t)(2 * HEXT_MAX + 1) * L.nzp * L.nxp * sizeof(float));
    if (born) {
        take(pl.dc2, fbytes);
        if (!pl.need_bwd) { // du^n, du^{n-1}
            take(pl.p[0], fbytes * pl.ns);
            take(pl.p[1], fbytes * pl.ns);
        }
    }
    take(pl.u[0], fbytes * pl.ns);
    take(pl.u[1], fbytes * pl.ns);
    if (pl.need_bwd) {
        take(pl.p[0], fbytes * pl.ns);
        take(pl.p[1], fbytes * pl.ns);
        if (!pl.snap) {
            take(pl.band, (size_t)pl.ns * pl.nt * L.nbandp * sizeof(float));
        } else {
            // levels 0..nt-2 are needed; segment j re-propagates levels
            // jK+1 .. min(jK+K-1, nt-2) from snapshot j (levels jK, jK-1)
            pl.snap_prec = o->snap_prec;
            pl.K = o->snap_interval > 0 ? o->snap_interval : (int)std::ceil(std::sqrt((double)pl.nt));
            pl.K = std::max(1, std::min(pl.K, pl.nt - 1));
            pl.nck = (pl.nt - 1 + pl.K - 1) / pl.K;
            pl.tr = make_tiling(L, pl.ns, STEP_FWD);
            const size_t esz = pl.snap_prec == FWI_SNAP_F32 ? 4 : 2;
            take(pl.snaps, (size_t)pl.nck * 2 * pl.ns * L.fstride * esz);
            if (pl.snap_prec != FWI_SNAP_F32) take(pl.snap_max, (size_t)pl.nck * 2 * pl.ns * sizeof(float));
            // K + 1 slots (K levels and u^{jK-1}); the two forward buffers
            // serve as slots 0 and 1
            if (pl.K + 1 > 2) take(pl.seg, fbytes * pl.ns * (size_t)(pl.K - 1));
        }
        take(pl.acc_g, (size_t)L.nzp * L.nxp * sizeof(float));
    }
    if (op == FWI_OP_GRADIENT || op == FWI_OP_GN_HVP || op == FWI_OP_MISFIT) take(pl.syn, (size_t)pl.ns * pl.nt * pl.nrec * sizeof(float));
    if (pl.need_bwd) take(pl.adj_t, (size_t)pl.ns * pl.nt * pl.nrec * sizeof(float));
    if (op == FWI_OP_GRADIENT || op == FWI_OP_ILLUMINATION)
        take(pl.acc_i, nphys * sizeof(float));
    if (pl.with_offh) take(pl.acc_h, (size_t)(pl.hmax + 1) * nphys * sizeof(float));
    // tables: src offsets, receiver CSR of the forward and backward tilings
    size_t t = 0;
    auto tk = [&](size_t &o2, size_t bytes) {
        o2 = t;
        t = align_up(t + bytes, 16);
    };
    tk(pl.tab_src, (size_t)pl.ns * sizeof(int));
    tk(pl.tab_srcij, (size_t)pl.ns * sizeof(int2));
    const size_t nent = (size_t)pl.ns * pl.nrec;
    // receiver tables: room for the tiling with the most tiles (any variant)
    const size_t mt = (size_t)max_tiles(L);
    tk(pl.tab_fptr, (mt * pl.ns + 1) * sizeof(int));
    tk(pl.tab_fent, std::max<size_t>(nent, 1) * sizeof(int2));
    if (pl.need_bwd || born) {
        tk(pl.tab_bptr, (mt * pl.ns + 1) * sizeof(int));
        tk(pl.tab_bent, std::max<size_t>(nent, 1) * sizeof(int2));
        tk(pl.tab_bshot, std::max<size_t>(nent, 1) * sizeof(int));
    }
    take(pl.tab, t);
    pl.total = off;
    return FWI_OK;
}

template <class T> T *at(void *ws, const Part &p) { return reinterpret_cast<T *>(static_cast<char *>(ws) + p.off); }
template <class T> T *at(void *ws, const Part &p, size_t extra)
{
    return reinterpret_cast<T *>(static_cast<char *>(ws) + p.off + extra);
}

void build_csr(const Plan &pl, const Tiling &t, const int *rec, std::vector<char> &buf, size_t ptr_off,
               size_t ent_off, size_t shot_off = (size_t)-1)
{
    const Lay2D &L = pl.L;
    const int ntiles = t.ntx * t.ntz;
    int *ptr = reinterpret_cast<int *>(buf.data() + ptr_off);
    int2 *ent = reinterpret_cast<int2 *>(buf.data() + ent_off);
    std::vector<int> cnt((size_t)ntiles * pl.ns + 1, 0);
    auto tile_of = [&](int s, int r, int &local) {
        const int *q = rec + 3 * ((long long)s * pl.nrec + r);
        const int i = q[0] + L.P, j = q[2] + L.P;
        const int tz = i / t.tz, tx = j / TX;
        local = (i - tz * t.tz) * TX + (j - tx * TX);
        return tz * t.ntx + tx;
    };
    for (int s = 0; s < pl.ns; ++s)
        for (int r = 0; r < pl.nrec; ++r) {
            int loc;
            const int tl = tile_of(s, r, loc);
            cnt[(size_t)tl * pl.ns + s + 1]++;
        }
    for (size_t k = 1; k < cnt.size(); ++k) cnt[k] += cnt[k - 1];
    std::memcpy(ptr, cnt.data(), cnt.size() * sizeof(int));
    std::vector<int> fill(cnt.begin(), cnt.end() - 1);
    for (int s = 0; s < pl.ns; ++s)
        for (int r = 0; r < pl.nrec; ++r) {
            int loc;
            const int tl = tile_of(s, r, loc);
            const int e = fill[(size_t)tl * pl.ns + s]++;
            ent[e] = make_int2(loc, r);
            if (shot_off != (size_t)-1) reinterpret_cast<int *>(buf.data() + shot_off)[e] = s;
        }
}

fwi_status upload_tables(const Plan &pl, const fwi_geometry *ge, void *ws, cudaStream_t st)
{
    std::vector<char> buf(pl.tab.bytes, 0);
    int *src = reinterpret_cast<int *>(buf.data() + pl.tab_src);
    int2 *srcij = reinterpret_cast<int2 *>(buf.data() + pl.tab_srcij);
    for (int s = 0; s < pl.ns; ++s) {
        const int *c = ge->src + 3 * s;
        src[s] = (int)fidx(pl.L, c[0] + pl.L.P, c[2] + pl.L.P);
        srcij[s] = make_int2(c[0] + pl.L.P, c[2] + pl.L.P);
    }
    if (pl.nrec > 0) {
        build_csr(pl, pl.tf, ge->rec, buf, pl.tab_fptr, pl.tab_fent);
        if (pl.need_bwd || pl.born) build_csr(pl, pl.tb, ge->rec, buf, pl.tab_bptr, pl.tab_bent, pl.tab_bshot);
    }
    cudaError_t e = cudaMemcpyAsync(at<char>(ws, pl.tab), buf.data(), buf.size(), cudaMemcpyHostToDevice, st);
    if (e != cudaSuccess) return cuda_fail(e, "upload of geometry tables");
    return FWI_OK;
}

// a caller's workspace: present, ALIGN-aligned, at least `need` bytes
fwi_status check_ws_bytes(void *ws, size_t ws_bytes, size_t need)
{
    if (!ws) return fail(FWI_ERR_INVALID_ARG, "workspace is NULL");
    if (reinterpret_cast<uintptr_t>(ws) % ALIGN != 0)
        return fail(FWI_ERR_INVALID_ARG, "workspace must be %zu-byte aligned", ALIGN);
    if (ws_bytes < need) return fail(FWI_ERR_NOMEM, "workspace of %zu bytes, need %zu", ws_bytes, need);
    return FWI_OK;
}

// the receivers' extent along x and mean row of one spread (nrec >= 1)
void spread_extent(const int *rec, int nrec, int &xmin, int &xmax, float &zmean)
{
    xmin = rec[2];
    xmax = rec[2];
    double zsum = 0;
    for (int r = 0; r < nrec; ++r) {
        const int *q = rec + 3 * r;
        xmin = std::min(xmin, q[2]);
        xmax = std::max(xmax, q[2]);
        zsum += q[0];
    }
    zmean = (float)(zsum / nrec);
}

fwi_status check_ws(const Plan &pl, void *ws, size_t ws_bytes)
{
    return check_ws_bytes(ws, ws_bytes, pl.total);
}

void prof_record(int k, cudaStream_t st)
{
    if (!t_prof) return;
    if (!t_ev[0])
        for (int i = 0; i < 4; ++i) cudaEventCreate(&t_ev[i]);
    if (t_capturing)
        cudaEventRecordWithFlags(t_ev[k], st, cudaEventRecordExternal);
    else
        cudaEventRecord(t_ev[k], st);
    if (k == 3) t_ev_recorded = true;
}

StepCommon make_common(const Plan &pl, const fwi_geometry *ge, void *ws, const Tiling &t)
{
    StepCommon c{};
    c.L = pl.L;
    c.c2 = at<float>(ws, pl.c2);
    c.damp = at<float>(ws, pl.damp);
    c.src_off = at<int>(ws, pl.tab, pl.tab_src);
    c.src_ij = at<int2>(ws, pl.tab, pl.tab_srcij);
    c.wav = ge->wavelet;
    c.src_scale = 1.0f; // dx^(2-ndim) in 2-D
    c.ns = pl.ns;
    c.nt = pl.nt;
    c.nrec = pl.nrec;
    c.ntx = t.ntx;
    c.ntz = t.ntz;
    c.status = at<int>(ws, pl.scal, 8);
    c.sched = at<int>(ws, pl.sched);
    c.chunk = t.chunk;
    return c;
}

// set-up shared by every propagation: status, tables, c2, zero fields
// (tables = false: the geometry tables are already in ws, as in a recorded
// graph, which cannot copy from pageable host memory)
fwi_status setup(const Plan &pl, const fwi_geometry *ge, const float *v, void *ws, cudaStream_t st,
                 bool tables = true)
{
    cudaError_t e;
    if ((e = cudaMemsetAsync(at<char>(ws, pl.scal), 0, pl.scal.bytes, st)) != cudaSuccess)
        return cuda_fail(e, "memset");
    if ((e = cudaMemsetAsync(at<char>(ws, pl.sched), 0, pl.sched.bytes, st)) != cudaSuccess)
        return cuda_fail(e, "memset");
    if (tables) {
        fwi_status s = upload_tables(pl, ge, ws, st);
        if (s != FWI_OK) return s;
    }
    if ((e = cudaMemsetAsync(at<char>(ws, pl.c2), 0, pl.c2.bytes, st)) != cudaSuccess) return cuda_fail(e, "memset");
    if ((e = cudaMemsetAsync(at<char>(ws, pl.damp), 0, pl.damp.bytes, st)) != cudaSuccess)
        return cuda_fail(e, "memset");
    if ((e = launch_prep_c2(pl.L, v, at<float>(ws, pl.c2), at<float>(ws, pl.damp), CFL_2D, at<int>(ws, pl.scal, 8),
                            st)) != cudaSuccess)
        return cuda_fail(e, "prep kernel");
    t_launch[2]++;
    for (int b = 0; b < 2; ++b)
        if ((e = cudaMemsetAsync(at<char>(ws, pl.u[b]), 0, pl.u[b].bytes, st)) != cudaSuccess)
            return cuda_fail(e, "memset");
    return FWI_OK;
}

// element count of one wavefield buffer (all shots)
inline long long field_elems(const Plan &pl) { return (long long)pl.ns * pl.L.fstride; }

fwi_status capture_snapshot(const Plan &pl, void *ws, int j, const float *u, const float *up, cudaStream_t st)
{
    const long long ne = field_elems(pl);
    cudaError_t e;
    if (pl.snap_prec == FWI_SNAP_F32) {
        float *dst = at<float>(ws, pl.snaps) + (size_t)j * 2 * ne;
        if ((e = cudaMemcpyAsync(dst, u, ne * sizeof(float), cudaMemcpyDeviceToDevice, st)) != cudaSuccess ||
            (e = cudaMemcpyAsync(dst + ne, up, ne * sizeof(float), cudaMemcpyDeviceToDevice, st)) != cudaSuccess)
            return cuda_fail(e, "snapshot copy");
        return FWI_OK;
    }
    float *mx = at<float>(ws, pl.snap_max) + (size_t)j * 2 * pl.ns;
    void *dst = at<char>(ws, pl.snaps) + (size_t)j * 2 * ne * 2;
    if ((e = launch_snap_absmax(u, up, pl.ns, pl.L.fstride, mx, st)) != cudaSuccess) return cuda_fail(e, "snapshot max");
    if ((e = launch_snap_encode(u, up, pl.ns, pl.L.fstride, mx, pl.snap_prec, dst, st)) != cudaSuccess)
        return cuda_fail(e, "snapshot encode");
    t_launch[2] += 2;
    return FWI_OK;
}

fwi_status restore_snapshot(const Plan &pl, void *ws, int j, float *u, float *up, cudaStream_t st)
{
    const long long ne = field_elems(pl);
    cudaError_t e;
    if (pl.snap_prec == FWI_SNAP_F32) {
        const float *src = at<float>(ws, pl.snaps) + (size_t)j * 2 * ne;
        if ((e = cudaMemcpyAsync(u, src, ne * sizeof(float), cudaMemcpyDeviceToDevice, st)) != cudaSuccess ||
            (e = cudaMemcpyAsync(up, src + ne, ne * sizeof(float), cudaMemcpyDeviceToDevice, st)) != cudaSuccess)
            return cuda_fail(e, "snapshot copy");
        return FWI_OK;
    }
    const float *mx = at<float>(ws, pl.snap_max) + (size_t)j * 2 * pl.ns;
    const void *src = at<char>(ws, pl.snaps) + (size_t)j * 2 * ne * 2;
    if ((e = launch_snap_decode(src, mx, pl.snap_prec, pl.ns, pl.L.fstride, u, up, st)) != cudaSuccess)
        return cuda_fail(e, "snapshot decode");
    t_launch[2]++;
    return FWI_OK;
}

// forward time loop n = 0..nt-1 of nm models at once (nm = 1: one model;
// nm > 1: one batched launch per time level, sponge checkpoints only). Model
// k's plan, geometry, workspace and outputs are pl[k], ge[k], ws[k], seis[k],
// acc_i[k], acc_h[k] (outputs may be null).
// Born time loop n = 0..nt-1: u and du = J dv advanced together (the du
// buffers are the adjoint-state buffers p), Born traces into dseis; with
// `save` the sponge checkpoint of u for a following adjoint pass
fwi_status run_born(const Plan &pl, const fwi_geometry *ge, void *ws, float *dseis, bool save, cudaStream_t st,
                    int he = 0)
{
    cudaError_t e;
    BornArgs a{};
    a.c = make_common(pl, ge, ws, pl.tb);
    a.dc2 = he > 0 ? nullptr : at<float>(ws, pl.dc2);
    a.dext = he > 0 ? at<float>(ws, pl.dext) : nullptr;
    a.band = save ? at<float>(ws, pl.band) : nullptr;
    a.dseis = (dseis && pl.nrec > 0) ? dseis : nullptr;
    a.rt.ptr = at<int>(ws, pl.tab, pl.tab_bptr);
    a.rt.ent = at<int2>(ws, pl.tab, pl.tab_bent);
    float *U[2] = {at<float>(ws, pl.u[0]), at<float>(ws, pl.u[1])};
    float *DU[2] = {at<float>(ws, pl.p[0]), at<float>(ws, pl.p[1])};
    for (int b = 0; b < 2; ++b)
        if ((e = cudaMemsetAsync(DU[b], 0, pl.p[b].bytes, st)) != cudaSuccess) return cuda_fail(e, "memset");
    int hx, hy, px, py;
    if (he > 0)
        ext_boxes(he, pl.tb, hx, hy, px, py);
    else
        step_boxes(STEP_BWD, pl.tb, hx, hy, px, py);
    CUtensorMap uh[2], up[2], dh[2], dp[2];
    for (int b = 0; b < 2; ++b)
        if (!encode_field_map(&uh[b], U[b], pl.L, pl.ns, hx, hy) || !encode_field_map(&up[b], U[b], pl.L, pl.ns, px, py) ||
            !encode_field_map(&dh[b], DU[b], pl.L, pl.ns, hx, hy) || !encode_field_map(&dp[b], DU[b], pl.L, pl.ns, px, py))
            return fail(FWI_ERR_CUDA, "cuTensorMapEncodeTiled failed for the wavefield buffers");
    for (int n = 0; n < pl.nt; ++n) {
        a.n = n;
        a.last = n == pl.nt - 1;
        a.tm_u = uh[n & 1];
        a.tm_du = dh[n & 1];
        a.tm_up = up[(n + 1) & 1];
        a.tm_dup = dp[(n + 1) & 1];
        a.uout = U[(n + 1) & 1];
        a.duout = DU[(n + 1) & 1];
        a.c.sched = at<int>(ws, pl.sched) + n;
        e = he > 0 ? launch_born_ext_step(a, pl.tb, he, st) : launch_born_step(a, pl.tb, st);
        if (e != cudaSuccess) return cuda_fail(e, "Born step");
        t_launch[0]++;
    }
    for (int b = 0; b < 2; ++b) {
        if ((e = launch_check_finite(U[b], (long long)pl.ns * pl.L.fstride, at<int>(ws, pl.scal, 8), st)) != cudaSuccess ||
            (e = launch_check_finite(DU[b], (long long)pl.ns * pl.L.fstride, at<int>(ws, pl.scal, 8), st)) != cudaSuccess)
            return cuda_fail(e, "finite check");
        t_launch[2] += 2;
    }
    return FWI_OK;
}

// (levels [n0, n1) only, and events around the step launches, when timing
// tile variants)
fwi_status run_forward_models(int nm, const Plan *pl, const fwi_geometry *const *ge, void *const *ws,
                              float *const *seis, bool save, float *const *acc_i, float *const *acc_h, int illum_utt,
                              cudaStream_t st, int n0 = 0, int n1 = -1, cudaEvent_t ev0 = nullptr,
                              cudaEvent_t ev1 = nullptr)
{
    cudaError_t e;
    std::vector<FwdArgs> a(nm);
    std::vector<Tiling> til(nm);
    std::vector<std::array<float *, 2>> U(nm);
    std::vector<std::array<CUtensorMap, 2>> mh(nm), mp(nm);
    const bool offh = pl[0].with_offh && acc_h[0];
    for (int k = 0; k < nm; ++k) {
        int hx, hy, px, py;
        step_boxes(offh ? STEP_FWD_OFFH : STEP_FWD, pl[k].tf, hx, hy, px, py);
        const Plan &p = pl[k];
        void *w = ws[k];
        if (acc_i[k] && (e = cudaMemsetAsync(acc_i[k], 0, p.acc_i.bytes, st)) != cudaSuccess)
            return cuda_fail(e, "memset");
        if (acc_h[k] && (e = cudaMemsetAsync(acc_h[k], 0, p.acc_h.bytes, st)) != cudaSuccess)
            return cuda_fail(e, "memset");
        a[k] = FwdArgs{};
        a[k].c = make_common(p, ge[k], w, p.tf);
        a[k].c.status = at<int>(ws[0], pl[0].scal, 8); // one status word per launch
        a[k].band = (save && !p.snap) ? at<float>(w, p.band) : nullptr;
        a[k].seis = (seis[k] && p.nrec > 0) ? seis[k] : nullptr;
        a[k].acc_illum = acc_i[k];
        a[k].acc_offh = acc_h[k];
        a[k].rt.ptr = at<int>(w, p.tab, p.tab_fptr);
        a[k].rt.ent = at<int2>(w, p.tab, p.tab_fent);
        a[k].illum_utt = illum_utt;
        a[k].hmax = p.hmax;
        til[k] = p.tf;
        U[k] = {at<float>(w, p.u[0]), at<float>(w, p.u[1])};
        for (int b = 0; b < 2; ++b)
            if (!encode_field_map(&mh[k][b], U[k][b], p.L, p.ns, hx, hy, p.tf.spi) ||
                !encode_field_map(&mp[k][b], U[k][b], p.L, p.ns, px, py, p.tf.spi))
                return fail(FWI_ERR_CUDA, "cuTensorMapEncodeTiled failed for the wavefield buffers");
    }
    const bool capture = nm == 1 && save && pl[0].snap;
    const int nt = pl[0].nt;
    if (n1 < 0) n1 = nt;
    if (ev0) cudaEventRecord(ev0, st);
    for (int n = n0; n < n1; ++n) {
        if (capture && n % pl[0].K == 0 && n <= nt - 2) {
            // snapshot n / K of the state (u^n, u^{n-1}) before step n
            fwi_status sc = capture_snapshot(pl[0], ws[0], n / pl[0].K, U[0][n & 1], U[0][(n + 1) & 1], st);
            if (sc != FWI_OK) return sc;
        }
        for (int k = 0; k < nm; ++k) {
            a[k].n = n;
            a[k].last = (n == nt - 1);
            a[k].tm_cur = mh[k][n & 1];
            a[k].tm_prev = mp[k][(n + 1) & 1];
            a[k].c.sched = at<int>(ws[0], pl[0].sched) + n;
            a[k].uin = U[k][n & 1];
            a[k].uout = U[k][(n + 1) & 1];
        }
        e = nm == 1 ? launch_fwd_step(a[0], til[0], offh, st) : launch_fwd_batch(a.data(), til.data(), nm, offh, st);
        if (e != cudaSuccess) return cuda_fail(e, "forward step");
        t_launch[0] += fwd_split(til[0], offh) ? 1 + nm : 1; // (split: one offset-Hessian sum per model)
    }
    if (ev1) cudaEventRecord(ev1, st);
    for (int k = 0; k < nm; ++k)
        for (int b = 0; b < 2; ++b) {
            if ((e = launch_check_finite(U[k][b], (long long)pl[k].ns * pl[k].L.fstride, at<int>(ws[k], pl[k].scal, 8),
                                         st)) != cudaSuccess)
                return cuda_fail(e, "finite check");
            t_launch[2]++;
        }
    return FWI_OK;
}

fwi_status run_forward(const Plan &pl, const fwi_geometry *ge, void *ws, float *seis, bool save,
                       float *acc_i, float *acc_h, int illum_utt, cudaStream_t st)
{
    return run_forward_models(1, &pl, &ge, &ws, &seis, save, &acc_i, &acc_h, illum_utt, st);
}

// Backward loop with snapshot checkpoints. For segment j = nck-1..0 (levels
// n_j = jK .. e_j = min(jK+K-1, nt-2)): restore (u^{n_j}, u^{n_j-1}) from
// snapshot j, re-run forward steps n_j..e_j into one slot per level, then
// run adjoint steps m = e_j+1 .. n_j+1. The re-run is the same plain forward
// step as the forward loop (no traces, no accumulators), so with F32
// snapshots it reproduces the forward's own fields; its step n also keeps
// the imaging factor q^n = Lhat u^n + f delta_s, in place of u^{n-1} (read
// only by the thread that then writes q^n there), and adjoint step m reads
// q^{m-1} instead of computing it from u^{m-1}. Step e_j computes q^{e_j}
// only.
fwi_status run_backward_segments(const Plan &pl, const fwi_geometry *ge, void *ws, BwdArgs &a, float *const U[2],
                                 float *const Pp[2], const CUtensorMap ph[2], const CUtensorMap pp[2], cudaStream_t st)
{
    cudaError_t e;
    const int K = pl.K;
    // slot i < K holds level n_j + i; slot K holds u^{n_j - 1}
    std::vector<float *> S(K + 1);
    for (int i = 0; i <= K; ++i)
        S[i] = i < 2 ? U[i] : at<float>(ws, pl.seg) + (size_t)(i - 2) * field_elems(pl);
    // the re-run writes only the padded model: the ghost frame of every slot
    // must read as zero
    for (int b = 0; b < 2; ++b)
        if ((e = cudaMemsetAsync(U[b], 0, pl.u[b].bytes, st)) != cudaSuccess) return cuda_fail(e, "memset");
    if (pl.seg.bytes && (e = cudaMemsetAsync(at<char>(ws, pl.seg), 0, pl.seg.bytes, st)) != cudaSuccess)
        return cuda_fail(e, "memset");
    int fhx, fhy, fpx, fpy, bhx, bhy, bpx, bpy;
    step_boxes(STEP_FWD, pl.tr, fhx, fhy, fpx, fpy);
    step_boxes(STEP_BWD, pl.tb, bhx, bhy, bpx, bpy);
    std::vector<CUtensorMap> fh(K + 1), fp(K + 1), bq(K + 1);
    for (int i = 0; i <= K; ++i)
        if (!encode_field_map(&fh[i], S[i], pl.L, pl.ns, fhx, fhy, pl.tr.spi) ||
            !encode_field_map(&fp[i], S[i], pl.L, pl.ns, fpx, fpy, pl.tr.spi) ||
            !encode_field_map(&bq[i], S[i], pl.L, pl.ns, bpx, bpy))
            return fail(FWI_ERR_CUDA, "cuTensorMapEncodeTiled failed for the segment buffers");
    auto qbuf = [&](int i) { return i == 0 ? K : i - 1; }; // slot of q^{n_j + i}
    FwdArgs f{};
    f.c = make_common(pl, ge, ws, pl.tr);
    f.hmax = -1;
    a.qin = 1;
    for (int j = pl.nck - 1; j >= 0; --j) {
        const int n0 = j * K, n1 = std::min(n0 + K - 1, pl.nt - 2);
        fwi_status sr = restore_snapshot(pl, ws, j, S[0], S[K], st);
        if (sr != FWI_OK) return sr;
        for (int n = n0; n <= n1; ++n) {
            const int i = n - n0;
            f.n = n;
            f.last = 0;
            f.tm_cur = fh[i];
            f.tm_prev = fp[qbuf(i)];
            f.uout = n < n1 ? S[i + 1] : nullptr;
            f.qout = S[qbuf(i)];
            f.c.sched = at<int>(ws, pl.sched) + 2 * pl.nt + n;
            if ((e = launch_fwd_step(f, pl.tr, false, st)) != cudaSuccess) return cuda_fail(e, "segment step");
            t_launch[1]++;
        }
        for (int m = n1 + 1; m >= n0 + 1; --m) {
            a.m = m;
            a.c.sched = at<int>(ws, pl.sched) + pl.nt + m;
            a.tm_ub = bq[qbuf(m - 1 - n0)];
            a.tm_pa = ph[(m + 1) & 1];
            a.tm_ua = pp[m & 1]; // not read without reconstruction
            a.tm_pb = pp[m & 1];
            a.ua = nullptr;
            a.pb = Pp[m & 1];
            if ((e = launch_bwd_step(a, pl.tb, st)) != cudaSuccess) return cuda_fail(e, "backward step");
            t_launch[1]++;
        }
    }
    if ((e = launch_check_finite(Pp[0], field_elems(pl), at<int>(ws, pl.scal, 8), st)) != cudaSuccess)
        return cuda_fail(e, "finite check");
    t_launch[2]++;
    return FWI_OK;
}

// backward time loop m = nt-1..1 of nm models at once (nm > 1: one batched
// launch per time level, sponge checkpoints only), adjoint source adj[k]
// [ns][nt][nrec] of model k
fwi_status run_backward_models(int nm, const Plan *pl, const fwi_geometry *const *ge, void *const *ws,
                               const float *const *adj, cudaStream_t st, int m_hi = -1, int m_lo = 1,
                               cudaEvent_t ev0 = nullptr, cudaEvent_t ev1 = nullptr, int he = 0,
                               float *acc_ext = nullptr)
{
    cudaError_t e;
    std::vector<BwdArgs> a(nm);
    std::vector<Tiling> til(nm);
    std::vector<std::array<float *, 2>> U(nm), Pp(nm);
    std::vector<std::array<CUtensorMap, 2>> uh(nm), up(nm), ph(nm), pp(nm);
    for (int k = 0; k < nm; ++k) {
        const Plan &p = pl[k];
        int hx, hy, px, py;
        if (he > 0)
            ext_boxes(he, p.tb, hx, hy, px, py);
        else
            step_boxes(STEP_BWD, p.tb, hx, hy, px, py);
        void *w = ws[k];
        for (int b = 0; b < 2; ++b)
            if ((e = cudaMemsetAsync(at<char>(w, p.p[b]), 0, p.p[b].bytes, st)) != cudaSuccess)
                return cuda_fail(e, "memset");
        if ((e = cudaMemsetAsync(at<char>(w, p.acc_g), 0, p.acc_g.bytes, st)) != cudaSuccess)
            return cuda_fail(e, "memset");
        a[k] = BwdArgs{};
        a[k].c = make_common(p, ge[k], w, p.tb);
        a[k].c.status = at<int>(ws[0], pl[0].scal, 8); // one status word per launch
        a[k].band = p.snap ? nullptr : at<float>(w, p.band);
        a[k].adj = nullptr;
        if (p.nrec > 0) {
            // adjoint source in the order of the backward receiver table: each
            // (tile, shot) reads one contiguous run per time level
            if ((e = launch_permute_adj(adj[k], at<int2>(w, p.tab, p.tab_bent), at<int>(w, p.tab, p.tab_bshot),
                                        p.ns * p.nrec, p.nt, p.nrec, at<float>(w, p.adj_t), st)) != cudaSuccess)
                return cuda_fail(e, "adjoint-source permutation");
            t_launch[2]++;
            a[k].adj = at<float>(w, p.adj_t);
        }
        a[k].nent = p.ns * p.nrec;
        a[k].acc_grad = at<float>(w, p.acc_g);
        a[k].rt.ptr = at<int>(w, p.tab, p.tab_bptr);
        a[k].rt.ent = at<int2>(w, p.tab, p.tab_bent);
        a[k].adj_scale = p.L.dx * p.L.dx;
        a[k].recon = p.snap ? 0 : 1;
        a[k].acc_ext = acc_ext;
        til[k] = p.tb;
        U[k] = {at<float>(w, p.u[0]), at<float>(w, p.u[1])};
        Pp[k] = {at<float>(w, p.p[0]), at<float>(w, p.p[1])};
        for (int b = 0; b < 2; ++b)
            if (!encode_field_map(&uh[k][b], U[k][b], p.L, p.ns, hx, hy) ||
                !encode_field_map(&up[k][b], U[k][b], p.L, p.ns, px, py) ||
                !encode_field_map(&ph[k][b], Pp[k][b], p.L, p.ns, hx, hy) ||
                !encode_field_map(&pp[k][b], Pp[k][b], p.L, p.ns, px, py))
                return fail(FWI_ERR_CUDA, "cuTensorMapEncodeTiled failed for the wavefield buffers");
    }
    if (nm == 1 && pl[0].snap) {
        float *U0[2] = {U[0][0], U[0][1]}, *P0[2] = {Pp[0][0], Pp[0][1]};
        CUtensorMap ph0[2] = {ph[0][0], ph[0][1]}, pp0[2] = {pp[0][0], pp[0][1]};
        return run_backward_segments(pl[0], ge[0], ws[0], a[0], U0, P0, ph0, pp0, st);
    }
    const int nt = pl[0].nt;
    if (m_hi < 0) m_hi = nt - 1;
    if (ev0) cudaEventRecord(ev0, st);
    for (int m = m_hi; m >= m_lo; --m) {
        for (int k = 0; k < nm; ++k) {
            a[k].m = m;
            a[k].c.sched = at<int>(ws[0], pl[0].sched) + nt + m;
            a[k].tm_ub = uh[k][(m - 1) & 1];
            a[k].tm_pa = ph[k][(m + 1) & 1];
            a[k].tm_ua = up[k][m & 1];
            a[k].tm_pb = pp[k][m & 1];
            a[k].ua = U[k][m & 1];
            a[k].pb = Pp[k][m & 1];
        }
        e = he > 0 ? launch_bwd_ext_step(a[0], til[0], he, st)
                   : (nm == 1 ? launch_bwd_step(a[0], til[0], st) : launch_bwd_batch(a.data(), til.data(), nm, st));
        if (e != cudaSuccess) return cuda_fail(e, "backward step");
        t_launch[1]++;
    }
    if (ev1) cudaEventRecord(ev1, st);
    for (int k = 0; k < nm; ++k) {
        if ((e = launch_check_finite(Pp[k][0], (long long)pl[k].ns * pl[k].L.fstride, at<int>(ws[k], pl[k].scal, 8),
                                     st)) != cudaSuccess)
            return cuda_fail(e, "finite check");
        t_launch[2]++;
    }
    return FWI_OK;
}

fwi_status run_backward(const Plan &pl, const fwi_geometry *ge, void *ws, const float *adj, cudaStream_t st)
{
    return run_backward_models(1, &pl, &ge, &ws, &adj, st);
}

// end of a call: read the status words of the call's models (one stream
// synchronisation), then the profile events
fwi_status finish_models(int nm, const Plan *pl, void *const *ws, cudaStream_t st)
{
    std::vector<int> status(nm, 0);
    cudaError_t e = cudaSuccess;
    for (int k = 0; k < nm && e == cudaSuccess; ++k)
        e = cudaMemcpyAsync(&status[k], at<int>(ws[k], pl[k].scal, 8), sizeof(int), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return cuda_fail(e, "status read-back");
    int any = 0;
    for (int k = 0; k < nm; ++k) any |= status[k];
    if (t_ev_recorded && t_prof) {
        float ms[3] = {0, 0, 0}, tot = 0;
        cudaEventElapsedTime(&ms[0], t_ev[0], t_ev[1]);
        cudaEventElapsedTime(&ms[1], t_ev[1], t_ev[2]);
        cudaEventElapsedTime(&tot, t_ev[0], t_ev[3]);
        t_times.forward_ms = ms[0];
        t_times.adjoint_ms = ms[1];
        t_times.other_ms = tot - ms[0] - ms[1];
        t_times.forward_launches = t_launch[0];
        t_times.adjoint_launches = t_launch[1];
        t_times.other_launches = t_launch[2];
    }
    if (any & ST_BAD_VELOCITY) return fail(FWI_ERR_INVALID_ARG, "velocity not finite and positive");
    if (any & ST_CFL) return fail(FWI_ERR_CFL, "v dt/dx above the stability limit %g", CFL_2D);
    if (any & ST_TIMEOUT) return fail(FWI_ERR_TIMEOUT, "a device wait timed out");
    if (any & ST_NONFINITE) return fail(FWI_ERR_UNSTABLE, "non-finite wavefield");
    t_err.clear();
    return FWI_OK;
}

fwi_status finish(const Plan &pl, void *ws, cudaStream_t st) { return finish_models(1, &pl, &ws, st); }

void begin_call(cudaStream_t st)
{
    t_launch[0] = t_launch[1] = t_launch[2] = 0;
    t_ev_recorded = false;
    prof_record(0, st);
}

// Device pointers of one model's gradient call (grad_pre, misfit, illum,
// offh may be null).
struct GradientIO {
    const float *v, *d_obs;
    float *grad, *grad_pre;
    double *misfit;
    float *illum, *offh;
};

// The whole preconditioned gradient of nm models (fwi_adjoint_gradient,
// fwi_batch_gradient): set-up, forward time loop, misfit and adjoint source,
// backward time loop, fold, illumination / offset-Hessian outputs and
// preconditioning. The time loops of all models run as one launch per level.
fwi_status gradient_models(int nm, const Plan *pl, const fwi_geometry *const *ge, const fwi_options *opts,
                           void *const *ws, const GradientIO *io, cudaStream_t st, bool tables = true,
                           cudaEvent_t input_ev = nullptr)
{
    fwi_status s;
    cudaError_t e;
    begin_call(st);
    std::vector<float *> acc_i(nm), acc_h(nm), syn(nm);
    for (int k = 0; k < nm; ++k) {
        if ((s = setup(pl[k], ge[k], io[k].v, ws[k], st, tables)) != FWI_OK) return s;
        acc_i[k] = at<float>(ws[k], pl[k].acc_i);
        acc_h[k] = pl[k].with_offh ? at<float>(ws[k], pl[k].acc_h) : nullptr;
        syn[k] = at<float>(ws[k], pl[k].syn);
    }
    if ((s = run_forward_models(nm, pl, ge, ws, syn.data(), true, acc_i.data(), acc_h.data(), opts->illum_mode, st)) !=
        FWI_OK)
        return s;
    prof_record(1, st);
    // the observed traces may still be arriving (uploaded on another stream
    // during the forward pass): wait for them here, before their first use
    if (input_ev != nullptr &&
        (e = cudaStreamWaitEvent(st, input_ev, t_capturing ? cudaEventWaitExternal : 0)) != cudaSuccess)
        return cuda_fail(e, "wait for the observed traces");
    for (int k = 0; k < nm; ++k) {
        double *J = at<double>(ws[k], pl[k].scal, 0);
        const long long nsamp = (long long)pl[k].ns * pl[k].nt * pl[k].nrec;
        if (nsamp == 0) continue;
        if ((e = launch_residual_ols(syn[k], io[k].d_obs, nsamp, opts->misfit == FWI_MISFIT_OLS ? J : nullptr, st)) !=
            cudaSuccess)
            return cuda_fail(e, "residual kernel");
        t_launch[2]++;
        if (opts->misfit == FWI_MISFIT_TIME_INTEGRAL) {
            if ((e = launch_time_integral(syn[k], pl[k].ns, pl[k].nt, pl[k].nrec, pl[k].L.dt, J, st)) != cudaSuccess)
                return cuda_fail(e, "time-integral kernel");
            t_launch[2]++;
        }
    }
    std::vector<const float *> adj(syn.begin(), syn.end());
    if ((s = run_backward_models(nm, pl, ge, ws, adj.data(), st)) != FWI_OK) return s;
    prof_record(2, st);
    for (int k = 0; k < nm; ++k) {
        const Plan &p = pl[k];
        void *w = ws[k];
        const GradientIO &o = io[k];
        if ((e = launch_fold_grad(p.L, at<float>(w, p.acc_g), 1, o.v, o.grad, st)) != cudaSuccess)
            return cuda_fail(e, "fold kernel");
        t_launch[2]++;
        // illumination: dt sum u^2, or (1/dt^3) sum (second difference)^2
        const float iscale = opts->illum_mode == FWI_ILLUM_U2 ? p.L.dt : 1.0f / (p.L.dt * p.L.dt * p.L.dt);
        float *ill_out = o.illum ? o.illum : acc_i[k]; // in place into group 0 when not requested
        const float *v6 = opts->hess_v6 ? o.v : nullptr;
        if ((e = launch_finish_accum(p.L, acc_i[k], 1, 1, iscale, ill_out, st, v6)) != cudaSuccess)
            return cuda_fail(e, "illumination output");
        t_launch[2]++;
        float *off_out = nullptr;
        if (acc_h[k]) {
            off_out = o.offh ? o.offh : acc_h[k];
            if ((e = launch_finish_accum(p.L, acc_h[k], 1, p.hmax + 1, p.L.dt, off_out, st, v6)) != cudaSuccess)
                return cuda_fail(e, "offset-Hessian output");
            t_launch[2]++;
        }
        if (o.grad_pre) {
            if (opts->precond == FWI_PRECOND_NONE) {
                if ((e = cudaMemcpyAsync(o.grad_pre, o.grad, (size_t)p.L.nz * p.L.nx * sizeof(float),
                                         cudaMemcpyDeviceToDevice, st)) != cudaSuccess)
                    return cuda_fail(e, "copy");
            } else {
                const bool ill = opts->precond == FWI_PRECOND_ILLUM;
                if ((e = launch_precond(p.L, o.grad, ill ? ill_out : off_out, ill ? 1 : 2, p.hmax, opts->eps,
                                        o.grad_pre, at<unsigned>(w, p.scal, 12), st)) != cudaSuccess)
                    return cuda_fail(e, "precondition kernel");
                t_launch[2] += 2;
            }
        }
        if (o.misfit &&
            (e = cudaMemcpyAsync(o.misfit, at<double>(w, p.scal, 0), sizeof(double), cudaMemcpyDeviceToDevice, st)) !=
                cudaSuccess)
            return cuda_fail(e, "copy");
    }
    prof_record(3, st);
    return FWI_OK;
}

// ---------------------------------------------------------------------- 3-D
// Stability limit of v dt / dx in 3-D: (v dt/dx)^2 * 3 * max|symbol| <= 4
// with the 1-D max|symbol| of the 2-D limit above.
constexpr float CFL_3D = FWI_CFL_LIMIT_3D;

fwi_status check_grid3(const fwi_grid *g)
{
    if (!g) return fail(FWI_ERR_INVALID_ARG, "grid is NULL");
    if (g->nz < 1 || g->ny < 1 || g->nx < 1)
        return fail(FWI_ERR_INVALID_ARG, "nz=%d ny=%d nx=%d must be >= 1", g->nz, g->ny, g->nx);
    if (g->nt < 2) return fail(FWI_ERR_INVALID_ARG, "nt=%d must be >= 2", g->nt);
    if (g->sponge < 1 || g->sponge > 64) return fail(FWI_ERR_INVALID_ARG, "sponge=%d outside 1..64", g->sponge);
    if (!(g->dx > 0.f) || !std::isfinite(g->dx)) return fail(FWI_ERR_INVALID_ARG, "dx must be > 0");
    if (!(g->dt > 0.f) || !std::isfinite(g->dt)) return fail(FWI_ERR_INVALID_ARG, "dt must be > 0");
    if (!(g->vref > 0.f) || !std::isfinite(g->vref)) return fail(FWI_ERR_INVALID_ARG, "vref must be > 0");
    if (!(g->refl > 0.f && g->refl < 1.f)) return fail(FWI_ERR_INVALID_ARG, "refl must be in (0,1)");
    return FWI_OK;
}

fwi_status check_geom3(const fwi_grid *g, const fwi_geometry *ge, bool coords)
{
    if (!ge) return fail(FWI_ERR_INVALID_ARG, "geometry is NULL");
    if (ge->nshots < 1) return fail(FWI_ERR_INVALID_ARG, "nshots=%d must be >= 1", ge->nshots);
    if (ge->nrec < 0) return fail(FWI_ERR_INVALID_ARG, "nrec=%d must be >= 0", ge->nrec);
    if ((long long)ge->nshots * ge->nrec >= (1LL << 31)) return fail(FWI_ERR_INVALID_ARG, "too many receivers");
    if (!coords) return FWI_OK;
    if (!ge->src) return fail(FWI_ERR_INVALID_ARG, "geometry.src is NULL");
    if (ge->nrec > 0 && !ge->rec) return fail(FWI_ERR_INVALID_ARG, "geometry.rec is NULL");
    if (!ge->wavelet) return fail(FWI_ERR_INVALID_ARG, "geometry.wavelet is NULL");
    auto inside = [&](const int *c) {
        return c[0] >= 0 && c[0] < g->nz && c[1] >= 0 && c[1] < g->ny && c[2] >= 0 && c[2] < g->nx;
    };
    for (int s = 0; s < ge->nshots; ++s) {
        const int *c = ge->src + 3 * s;
        if (!inside(c))
            return fail(FWI_ERR_INVALID_ARG, "source of shot %d at (%d,%d,%d) outside the model", s, c[0], c[1], c[2]);
        for (int r = 0; r < ge->nrec; ++r) {
            const int *q = ge->rec + 3 * ((long long)s * ge->nrec + r);
            if (!inside(q))
                return fail(FWI_ERR_INVALID_ARG, "receiver %d of shot %d at (%d,%d,%d) outside the model", r, s, q[0],
                            q[1], q[2]);
        }
    }
    return FWI_OK;
}

Lay3D make_layout3(const fwi_grid *g)
{
    Lay3D L{};
    L.nz = g->nz;
    L.ny = g->ny;
    L.nx = g->nx;
    L.P = g->sponge;
    L.nzp = g->nz + 2 * g->sponge;
    L.nyp = g->ny + 2 * g->sponge;
    L.nxp = g->nx + 2 * g->sponge;
    L.pitch = (int)align_up((size_t)(GXL + L.nxp + GXR), 32);
    L.rows = L.nyp + 2 * GY;
    L.planes = L.nzp + 2 * GZ;
    L.plane = (long long)L.rows * L.pitch;
    L.fstride = (long long)align_up((size_t)(L.planes * L.plane), 64);
    L.dt = g->dt;
    L.dx = g->dx;
    const double etamax = 3.0 * g->vref * std::log(1.0 / g->refl) / (2.0 * g->sponge * g->dx);
    L.etamax_dt = (float)(etamax * g->dt);
    L.inv_p2 = (float)(1.0 / ((double)g->sponge * g->sponge));
    return L;
}

// One 3-D call: the shots are modelled in groups of G (opts->shot_group), each
// group in the same workspace; accumulators and the misfit sum over groups.
struct Plan3 {
    Lay3D L;
    int ns_all = 0, G = 0, nt = 0, nrec = 0, op = 0;
    int hmax = -1; // offsets of the offset Hessian (gradient, offset-Hessian diagonal), -1: none
    bool need_bwd = false;
    Tiling3 tf{}, tb{};
    int vf = 0, vb = 0; // step variants (autotuned per shape, else the defaults)
    Part scal, sched, c2, damp, u[2], p[2], syn, acc_i, acc_h, acc_g, tab, snaps, snap_max, seg;
    size_t tab_src = 0, tab_ptr = 0, tab_ent = 0, tab_zr = 0;
    int snap_prec = FWI_SNAP_F32, K = 0, nck = 0;
    size_t total = 0;
};

fwi_status make_plan3(const fwi_grid *g, const fwi_geometry *ge, const fwi_options *o, int op, bool coords,
                      Plan3 &pl)
{
    fwi_status st;
    if ((st = check_grid3(g)) != FWI_OK) return st;
    if ((st = check_geom3(g, ge, coords)) != FWI_OK) return st;
    if ((st = check_opts(o, op)) != FWI_OK) return st;
    if (op != FWI_OP_FORWARD && op != FWI_OP_FORWARD_SAVE && op != FWI_OP_GRADIENT && op != FWI_OP_ILLUMINATION &&
        op != FWI_OP_OFFSET_HESSIAN)
        return fail(FWI_ERR_INVALID_ARG, "3-D grids support forward modelling (with or without checkpoints for "
                                         "fwi_adjoint_apply), gradients, illumination and the offset Hessian");
    if (op == FWI_OP_OFFSET_HESSIAN && o->hmax < 0)
        return fail(FWI_ERR_INVALID_ARG, "the offset-Hessian diagonal needs hmax >= 0");
    const bool ckpts = op == FWI_OP_GRADIENT || op == FWI_OP_FORWARD_SAVE;
    if (ckpts && (!o || o->ckpt != FWI_CKPT_SNAPSHOT))
        return fail(FWI_ERR_INVALID_ARG, "3-D gradients and fwi_forward(save = 1) need ckpt = FWI_CKPT_SNAPSHOT "
                                         "(a per-level sponge band of a 3-D grid does not fit)");
    if (op == FWI_OP_FORWARD_SAVE && o->shot_group > 0 && o->shot_group < ge->nshots)
        return fail(FWI_ERR_INVALID_ARG, "3-D fwi_forward(save = 1) keeps the snapshots of every shot for "
                                         "fwi_adjoint_apply: shot_group must be 0 or >= nshots");
    pl.L = make_layout3(g);
    pl.hmax = (op == FWI_OP_GRADIENT || op == FWI_OP_OFFSET_HESSIAN) ? o->hmax : -1;
    pl.op = op;
    pl.nt = g->nt;
    pl.ns_all = ge->nshots;
    pl.nrec = ge->nrec;
    pl.G = (o && o->shot_group > 0 && o->shot_group < ge->nshots) ? o->shot_group : ge->nshots;
    pl.need_bwd = ckpts; // forward-with-checkpoints has the gradient's layout
    const Lay3D &L = pl.L;
    pl.vf = step3_variant_for(L, pl.G, false);
    pl.vb = step3_variant_for(L, pl.G, true);
    pl.tf = make_tiling3(L, pl.G, false, pl.vf, step3_segments_for(L, pl.G, false));
    pl.tb = make_tiling3(L, pl.G, true, pl.vb, step3_segments_for(L, pl.G, true));
    size_t off = 0;
    auto take = [&](Part &p, size_t bytes) {
        p.off = off;
        p.bytes = bytes;
        off = align_up(off + bytes);
    };
    const size_t fbytes = (size_t)L.fstride * sizeof(float);
    const size_t nphys = (size_t)L.nz * L.ny * L.nx;
    take(pl.scal, 256);
    take(pl.sched, (size_t)3 * pl.nt * sizeof(int));
    take(pl.c2, fbytes);
    take(pl.damp, fbytes);
    take(pl.u[0], fbytes * pl.G);
    take(pl.u[1], fbytes * pl.G);
    if (op != FWI_OP_FORWARD) take(pl.acc_i, nphys * sizeof(float));
    if (pl.hmax >= 0) take(pl.acc_h, (size_t)(pl.hmax + 1) * nphys * sizeof(float));
    if (pl.need_bwd) {
        take(pl.p[0], fbytes * pl.G);
        take(pl.p[1], fbytes * pl.G);
        take(pl.syn, (size_t)pl.G * pl.nt * pl.nrec * sizeof(float));
        take(pl.acc_g, (size_t)L.nzp * L.nyp * L.nxp * sizeof(float));
        pl.snap_prec = o->snap_prec;
        pl.K = o->snap_interval > 0 ? o->snap_interval : (int)std::ceil(std::sqrt((double)pl.nt));
        pl.K = std::max(1, std::min(pl.K, pl.nt - 1));
        pl.nck = (pl.nt - 1 + pl.K - 1) / pl.K;
        const size_t esz = pl.snap_prec == FWI_SNAP_F32 ? 4 : 2;
        take(pl.snaps, (size_t)pl.nck * 2 * pl.G * L.fstride * esz);
        if (pl.snap_prec != FWI_SNAP_F32) take(pl.snap_max, (size_t)pl.nck * 2 * pl.G * sizeof(float));
        if (pl.K + 1 > 2) take(pl.seg, fbytes * pl.G * (size_t)(pl.K - 1));
    }
    const size_t ntiles = (size_t)pl.tf.nty * pl.tf.ntx;
    size_t t = 0;
    auto tk = [&](size_t &o2, size_t bytes) {
        o2 = t;
        t = align_up(t + bytes, 16);
    };
    tk(pl.tab_src, (size_t)pl.G * sizeof(int4));
    tk(pl.tab_ptr, (ntiles * pl.G + 1) * sizeof(int));
    tk(pl.tab_ent, std::max<size_t>((size_t)pl.G * pl.nrec, 1) * sizeof(int4));
    tk(pl.tab_zr, ntiles * pl.G * sizeof(int2));
    take(pl.tab, t);
    pl.total = off;
    return FWI_OK;
}

// geometry tables of shots [s0, s0 + g) of the call
fwi_status upload_tables3(const Plan3 &pl, const fwi_geometry *ge, int s0, int g, void *ws, cudaStream_t st)
{
    const Lay3D &L = pl.L;
    std::vector<char> buf(pl.tab.bytes, 0);
    int4 *src = reinterpret_cast<int4 *>(buf.data() + pl.tab_src);
    for (int s = 0; s < g; ++s) {
        const int *c = ge->src + 3 * (s0 + s);
        src[s] = make_int4(c[0] + L.P, c[1] + L.P, c[2] + L.P, 0);
    }
    const int ntiles = pl.tf.nty * pl.tf.ntx;
    int *ptr = reinterpret_cast<int *>(buf.data() + pl.tab_ptr);
    int4 *ent = reinterpret_cast<int4 *>(buf.data() + pl.tab_ent);
    int2 *zr = reinterpret_cast<int2 *>(buf.data() + pl.tab_zr);
    // entries of (tile, shot) in tile-major order, sorted by plane in each
    struct E {
        int key, plane, loc, r;
    };
    std::vector<E> es;
    es.reserve((size_t)g * pl.nrec);
    for (int s = 0; s < g; ++s)
        for (int r = 0; r < pl.nrec; ++r) {
            const int *q = ge->rec + 3 * ((long long)(s0 + s) * pl.nrec + r);
            const int i = q[0] + L.P, k = q[1] + L.P, j = q[2] + L.P;
            const int ty = k / TY3, tx = j / TX;
            es.push_back(E{(ty * pl.tf.ntx + tx) * g + s, i, (k - ty * TY3) * TX + (j - tx * TX), r});
        }
    std::stable_sort(es.begin(), es.end(), [](const E &a, const E &b) {
        return a.key != b.key ? a.key < b.key : a.plane < b.plane;
    });
    for (int k = 0; k < ntiles * g; ++k) zr[k] = make_int2(1, 0);
    size_t e = 0;
    for (int key = 0; key < ntiles * g; ++key) {
        ptr[key] = (int)e;
        while (e < es.size() && es[e].key == key) {
            ent[e] = make_int4(es[e].plane, es[e].loc, es[e].r, 0);
            if (zr[key].y < zr[key].x) zr[key] = make_int2(es[e].plane, es[e].plane);
            zr[key].x = std::min(zr[key].x, es[e].plane);
            zr[key].y = std::max(zr[key].y, es[e].plane);
            ++e;
        }
    }
    ptr[ntiles * g] = (int)e;
    cudaError_t err = cudaMemcpyAsync(at<char>(ws, pl.tab), buf.data(), buf.size(), cudaMemcpyHostToDevice, st);
    if (err != cudaSuccess) return cuda_fail(err, "upload of geometry tables");
    return FWI_OK;
}

Step3Common make_common3(const Plan3 &pl, const fwi_geometry *ge, int s0, int g, void *ws, const Tiling3 &t)
{
    Step3Common c{};
    c.L = pl.L;
    c.c2 = at<float>(ws, pl.c2);
    c.damp = at<float>(ws, pl.damp);
    c.src = at<int4>(ws, pl.tab, pl.tab_src);
    c.wav = ge->wavelet + (size_t)s0 * pl.nt;
    c.src_scale = 1.0f / pl.L.dx; // dx^(2 - 3)
    c.ns = g;
    c.nt = pl.nt;
    c.nrec = pl.nrec;
    c.nty = t.nty;
    c.ntx = t.ntx;
    c.nseg = t.nseg;
    c.segl = t.segl;
    c.status = at<int>(ws, pl.scal, 8);
    c.sched = at<int>(ws, pl.sched);
    return c;
}

Rec3Table rec_table3(const Plan3 &pl, void *ws)
{
    return Rec3Table{at<int>(ws, pl.tab, pl.tab_ptr), at<int4>(ws, pl.tab, pl.tab_ent), at<int2>(ws, pl.tab, pl.tab_zr)};
}

// point- and halo-box maps of a buffer of g 3-D fields
fwi_status maps3(const Plan3 &pl, const float *buf, int g, CUtensorMap *halo, CUtensorMap *pt)
{
    if ((halo && !encode_field_map3(halo, buf, pl.L, g, TX + 2 * RADIUS, TY3 + 2 * RADIUS)) ||
        (pt && !encode_field_map3(pt, buf, pl.L, g, TX, TY3)))
        return fail(FWI_ERR_CUDA, "cuTensorMapEncodeTiled failed for a 3-D buffer");
    return FWI_OK;
}

fwi_status snap3_capture(const Plan3 &pl, void *ws, int g, int j, const float *u, const float *up, cudaStream_t st)
{
    const long long ne = (long long)g * pl.L.fstride;
    cudaError_t e;
    if (pl.snap_prec == FWI_SNAP_F32) {
        float *dst = at<float>(ws, pl.snaps) + (size_t)j * 2 * ne;
        if ((e = cudaMemcpyAsync(dst, u, ne * sizeof(float), cudaMemcpyDeviceToDevice, st)) != cudaSuccess ||
            (e = cudaMemcpyAsync(dst + ne, up, ne * sizeof(float), cudaMemcpyDeviceToDevice, st)) != cudaSuccess)
            return cuda_fail(e, "snapshot copy");
        return FWI_OK;
    }
    float *mx = at<float>(ws, pl.snap_max) + (size_t)j * 2 * g;
    void *dst = at<char>(ws, pl.snaps) + (size_t)j * 2 * ne * 2;
    if ((e = launch_snap_absmax(u, up, g, pl.L.fstride, mx, st)) != cudaSuccess) return cuda_fail(e, "snapshot max");
    if ((e = launch_snap_encode(u, up, g, pl.L.fstride, mx, pl.snap_prec, dst, st)) != cudaSuccess)
        return cuda_fail(e, "snapshot encode");
    t_launch[2] += 2;
    return FWI_OK;
}

fwi_status snap3_restore(const Plan3 &pl, void *ws, int g, int j, float *u, float *up, cudaStream_t st)
{
    const long long ne = (long long)g * pl.L.fstride;
    cudaError_t e;
    if (pl.snap_prec == FWI_SNAP_F32) {
        const float *src = at<float>(ws, pl.snaps) + (size_t)j * 2 * ne;
        if ((e = cudaMemcpyAsync(u, src, ne * sizeof(float), cudaMemcpyDeviceToDevice, st)) != cudaSuccess ||
            (e = cudaMemcpyAsync(up, src + ne, ne * sizeof(float), cudaMemcpyDeviceToDevice, st)) != cudaSuccess)
            return cuda_fail(e, "snapshot copy");
        return FWI_OK;
    }
    const float *mx = at<float>(ws, pl.snap_max) + (size_t)j * 2 * g;
    const void *src = at<char>(ws, pl.snaps) + (size_t)j * 2 * ne * 2;
    if ((e = launch_snap_decode(src, mx, pl.snap_prec, g, pl.L.fstride, u, up, st)) != cudaSuccess)
        return cuda_fail(e, "snapshot decode");
    t_launch[2]++;
    return FWI_OK;
}

// forward time loop of one shot group [s0, s0 + g): traces into seis (the
// group's rows) or null, illumination into acc_i or null, the offset-Hessian
// sums of offsets 0..pl.hmax into acc_h or null, snapshots if `save`; levels
// [n_begin, n_end) (n_end < 0: to nt), events ea / eb (if given) recorded
// around the step launches
fwi_status run_forward3(const Plan3 &pl, const fwi_geometry *ge, int s0, int g, void *ws, float *seis,
                        float *acc_i, float *acc_h, int illum_utt, bool save, cudaStream_t st, int n_begin = 0,
                        int n_end = -1, cudaEvent_t ea = nullptr, cudaEvent_t eb = nullptr)
{
    cudaError_t e;
    for (int b = 0; b < 2; ++b)
        if ((e = cudaMemsetAsync(at<char>(ws, pl.u[b]), 0, (size_t)g * pl.L.fstride * sizeof(float), st)) !=
            cudaSuccess)
            return cuda_fail(e, "memset");
    if ((e = cudaMemsetAsync(at<char>(ws, pl.sched), 0, pl.sched.bytes, st)) != cudaSuccess)
        return cuda_fail(e, "memset");
    Fwd3Args a{};
    a.c = make_common3(pl, ge, s0, g, ws, pl.tf);
    a.seis = (seis && pl.nrec > 0) ? seis : nullptr;
    a.acc_illum = acc_i;
    a.rt = rec_table3(pl, ws);
    a.illum_utt = illum_utt;
    float *U[2] = {at<float>(ws, pl.u[0]), at<float>(ws, pl.u[1])};
    CUtensorMap mh[2], mp[2];
    fwi_status s;
    for (int b = 0; b < 2; ++b)
        if ((s = maps3(pl, U[b], g, &mh[b], &mp[b])) != FWI_OK) return s;
    if ((s = maps3(pl, at<float>(ws, pl.c2), 1, nullptr, &a.tm_c2)) != FWI_OK) return s;
    if ((s = maps3(pl, at<float>(ws, pl.damp), 1, nullptr, &a.tm_damp)) != FWI_OK) return s;
    if (n_end < 0) n_end = pl.nt;
    if (acc_h && (n_begin != 0 || n_end != pl.nt)) return fail(FWI_ERR_INVALID_ARG, "offset-Hessian sums need every level");
    if (ea && (e = cudaEventRecord(ea, st)) != cudaSuccess) return cuda_fail(e, "cudaEventRecord");
    for (int n = n_begin; n < n_end; ++n) {
        if (save && n % pl.K == 0 && n <= pl.nt - 2)
            if ((s = snap3_capture(pl, ws, g, n / pl.K, U[n & 1], U[(n + 1) & 1], st)) != FWI_OK) return s;
        a.n = n;
        a.last = n == pl.nt - 1;
        a.tm_u = mh[n & 1];
        a.tm_upt = mp[n & 1];
        a.tm_prev = mp[(n + 1) & 1];
        a.uin = U[n & 1];
        a.uout = U[(n + 1) & 1];
        a.c.sched = at<int>(ws, pl.sched) + n;
        if ((e = launch_fwd3d(a, pl.tf, pl.vf, st)) != cudaSuccess) return cuda_fail(e, "3-D forward step");
        t_launch[0]++;
        // after an even step n the buffers hold u^n (overwritten by step n + 1)
        // and u^{n+1} (written by step n when n <= nt - 2): both levels are
        // summed in one launch; u^0 = 0 adds nothing
        if (acc_h && n % 2 == 0) {
            const float *lo = n > 0 ? U[n & 1] : nullptr, *hi = n + 1 <= pl.nt - 1 ? U[(n + 1) & 1] : nullptr;
            if ((e = launch_offh3d(lo, hi, pl.L, g, pl.hmax, acc_h, st)) != cudaSuccess)
                return cuda_fail(e, "3-D offset-Hessian sums");
            t_launch[0]++;
        }
    }
    if (eb && (e = cudaEventRecord(eb, st)) != cudaSuccess) return cuda_fail(e, "cudaEventRecord");
    for (int b = 0; b < 2; ++b) {
        if ((e = launch_check_finite(U[b], (long long)g * pl.L.fstride, at<int>(ws, pl.scal, 8), st)) != cudaSuccess)
            return cuda_fail(e, "finite check");
        t_launch[2]++;
    }
    return FWI_OK;
}

// backward loop of one shot group from its snapshots (as in 2-D: segment by
// segment, last first, re-propagated then back-propagated); adj: the group's
// adjoint source [g][nt][nrec]
fwi_status run_backward3(const Plan3 &pl, const fwi_geometry *ge, int s0, int g, void *ws, const float *adj,
                         cudaStream_t st)
{
    cudaError_t e;
    fwi_status s;
    const int K = pl.K;
    const size_t gbytes = (size_t)g * pl.L.fstride * sizeof(float);
    std::vector<float *> S(K + 1);
    for (int i = 0; i <= K; ++i)
        S[i] = i < 2 ? at<float>(ws, pl.u[i]) : at<float>(ws, pl.seg) + (size_t)(i - 2) * g * pl.L.fstride;
    for (int i = 0; i <= K; ++i)
        if ((e = cudaMemsetAsync(S[i], 0, gbytes, st)) != cudaSuccess) return cuda_fail(e, "memset");
    float *Pp[2] = {at<float>(ws, pl.p[0]), at<float>(ws, pl.p[1])};
    for (int b = 0; b < 2; ++b)
        if ((e = cudaMemsetAsync(Pp[b], 0, gbytes, st)) != cudaSuccess) return cuda_fail(e, "memset");
    std::vector<CUtensorMap> sh(K + 1), sp(K + 1);
    for (int i = 0; i <= K; ++i)
        if ((s = maps3(pl, S[i], g, &sh[i], &sp[i])) != FWI_OK) return s;
    CUtensorMap ph[2], pp[2], c2m, dm;
    for (int b = 0; b < 2; ++b)
        if ((s = maps3(pl, Pp[b], g, &ph[b], &pp[b])) != FWI_OK) return s;
    if ((s = maps3(pl, at<float>(ws, pl.c2), 1, nullptr, &c2m)) != FWI_OK) return s;
    if ((s = maps3(pl, at<float>(ws, pl.damp), 1, nullptr, &dm)) != FWI_OK) return s;
    Fwd3Args f{};
    f.c = make_common3(pl, ge, s0, g, ws, pl.tf);
    f.rt = rec_table3(pl, ws);
    f.tm_c2 = c2m;
    f.tm_damp = dm;
    Bwd3Args a{};
    a.c = make_common3(pl, ge, s0, g, ws, pl.tb);
    a.rt = rec_table3(pl, ws);
    a.adj = pl.nrec > 0 ? adj : nullptr;
    a.acc_grad = at<float>(ws, pl.acc_g);
    a.adj_scale = pl.L.dx * pl.L.dx;
    a.tm_c2 = c2m;
    a.tm_damp = dm;
    if ((e = cudaMemsetAsync(at<char>(ws, pl.sched), 0, pl.sched.bytes, st)) != cudaSuccess)
        return cuda_fail(e, "memset");
    // Segment j: S[0] = u^{n0}, S[K] = u^{n0-1} from the snapshots; the
    // re-propagation's step n (levels n0 .. n1) reads u^n (S[n - n0]) and
    // u^{n-1}, writes u^{n+1} (S[n - n0 + 1]; not at n1) and, in place of
    // u^{n-1}, which nothing reads after it, the imaging factor
    // q^n = Lhat u^n + f delta_s / dx of the backward step n + 1.
    auto qbuf = [&](int i) { return i == 0 ? K : i - 1; }; // buffer of q^{n0 + i}
    for (int j = pl.nck - 1; j >= 0; --j) {
        const int n0 = j * K, n1 = std::min(n0 + K - 1, pl.nt - 2);
        if ((s = snap3_restore(pl, ws, g, j, S[0], S[K], st)) != FWI_OK) return s;
        for (int n = n0; n <= n1; ++n) {
            const int i = n - n0;
            f.n = n;
            f.last = 0;
            f.tm_u = sh[i];
            f.tm_upt = sp[i];
            f.tm_prev = sp[qbuf(i)];
            f.uin = S[i];
            f.uout = n < n1 ? S[i + 1] : nullptr;
            f.qout = S[qbuf(i)];
            f.c.sched = at<int>(ws, pl.sched) + 2 * pl.nt + n;
            if ((e = launch_fwd3d(f, pl.tf, pl.vf, st)) != cudaSuccess) return cuda_fail(e, "3-D segment step");
            t_launch[1]++;
        }
        for (int m = n1 + 1; m >= n0 + 1; --m) {
            a.m = m;
            a.tm_q = sp[qbuf(m - 1 - n0)];
            a.tm_p = ph[(m + 1) & 1];
            a.tm_ppt = pp[(m + 1) & 1];
            a.tm_pb = pp[m & 1];
            a.pin = Pp[(m + 1) & 1];
            a.pb = Pp[m & 1];
            a.c.sched = at<int>(ws, pl.sched) + pl.nt + m;
            if ((e = launch_bwd3d(a, pl.tb, pl.vb, st)) != cudaSuccess) return cuda_fail(e, "3-D backward step");
            t_launch[1]++;
        }
    }
    if ((e = launch_check_finite(Pp[0], (long long)g * pl.L.fstride, at<int>(ws, pl.scal, 8), st)) != cudaSuccess)
        return cuda_fail(e, "finite check");
    t_launch[2]++;
    return FWI_OK;
}

// nlev backward steps of the first group, levels nt-1 downwards, on the
// group's fields as they are (the autotuner's timing; events ea / eb around
// the launches). The imaging sum is overwritten by the next call's set-up.
fwi_status time_backward3(const Plan3 &pl, const fwi_geometry *ge, void *ws, int nlev, cudaStream_t st,
                          cudaEvent_t ea, cudaEvent_t eb)
{
    cudaError_t e;
    fwi_status s;
    const int g = pl.G;
    float *U[2] = {at<float>(ws, pl.u[0]), at<float>(ws, pl.u[1])};
    float *Pp[2] = {at<float>(ws, pl.p[0]), at<float>(ws, pl.p[1])};
    CUtensorMap uh[2], up[2], ph[2], pp[2];
    for (int b = 0; b < 2; ++b)
        if ((s = maps3(pl, U[b], g, &uh[b], &up[b])) != FWI_OK || (s = maps3(pl, Pp[b], g, &ph[b], &pp[b])) != FWI_OK)
            return s;
    Bwd3Args a{};
    a.c = make_common3(pl, ge, 0, g, ws, pl.tb);
    a.rt = rec_table3(pl, ws);
    a.adj = pl.nrec > 0 ? at<float>(ws, pl.syn) : nullptr;
    a.acc_grad = at<float>(ws, pl.acc_g);
    a.adj_scale = pl.L.dx * pl.L.dx;
    if ((s = maps3(pl, at<float>(ws, pl.c2), 1, nullptr, &a.tm_c2)) != FWI_OK) return s;
    if ((s = maps3(pl, at<float>(ws, pl.damp), 1, nullptr, &a.tm_damp)) != FWI_OK) return s;
    if ((e = cudaMemsetAsync(at<char>(ws, pl.sched), 0, pl.sched.bytes, st)) != cudaSuccess)
        return cuda_fail(e, "memset");
    if ((e = cudaEventRecord(ea, st)) != cudaSuccess) return cuda_fail(e, "cudaEventRecord");
    for (int m = pl.nt - 1; m >= 1 && m > pl.nt - 1 - nlev; --m) {
        a.m = m;
        a.tm_q = up[(m - 1) & 1]; // (timing only: any field as the imaging factor)
        a.tm_p = ph[(m + 1) & 1];
        a.tm_ppt = pp[(m + 1) & 1];
        a.tm_pb = pp[m & 1];
        a.pin = Pp[(m + 1) & 1];
        a.pb = Pp[m & 1];
        a.c.sched = at<int>(ws, pl.sched) + pl.nt + m;
        if ((e = launch_bwd3d(a, pl.tb, pl.vb, st)) != cudaSuccess) return cuda_fail(e, "3-D backward step");
    }
    if ((e = cudaEventRecord(eb, st)) != cudaSuccess) return cuda_fail(e, "cudaEventRecord");
    return FWI_OK;
}

fwi_status setup3(const Plan3 &pl, const float *v, void *ws, cudaStream_t st)
{
    cudaError_t e;
    if ((e = cudaMemsetAsync(at<char>(ws, pl.scal), 0, pl.scal.bytes, st)) != cudaSuccess) return cuda_fail(e, "memset");
    if ((e = cudaMemsetAsync(at<char>(ws, pl.c2), 0, pl.c2.bytes, st)) != cudaSuccess) return cuda_fail(e, "memset");
    if ((e = cudaMemsetAsync(at<char>(ws, pl.damp), 0, pl.damp.bytes, st)) != cudaSuccess)
        return cuda_fail(e, "memset");
    if ((e = launch_prep3d(pl.L, v, at<float>(ws, pl.c2), at<float>(ws, pl.damp), CFL_3D, at<int>(ws, pl.scal, 8),
                           st)) != cudaSuccess)
        return cuda_fail(e, "prep kernel");
    t_launch[2]++;
    if (pl.acc_i.bytes && (e = cudaMemsetAsync(at<char>(ws, pl.acc_i), 0, pl.acc_i.bytes, st)) != cudaSuccess)
        return cuda_fail(e, "memset");
    if (pl.acc_h.bytes && (e = cudaMemsetAsync(at<char>(ws, pl.acc_h), 0, pl.acc_h.bytes, st)) != cudaSuccess)
        return cuda_fail(e, "memset");
    if (pl.acc_g.bytes && (e = cudaMemsetAsync(at<char>(ws, pl.acc_g), 0, pl.acc_g.bytes, st)) != cudaSuccess)
        return cuda_fail(e, "memset");
    return FWI_OK;
}

fwi_status finish3(const Plan3 &pl, void *ws, cudaStream_t st)
{
    int status = 0;
    cudaError_t e = cudaMemcpyAsync(&status, at<int>(ws, pl.scal, 8), sizeof(int), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return cuda_fail(e, "status read-back");
    if (t_ev_recorded && t_prof) {
        float ms[3] = {0, 0, 0}, tot = 0;
        cudaEventElapsedTime(&ms[0], t_ev[0], t_ev[1]);
        cudaEventElapsedTime(&ms[1], t_ev[1], t_ev[2]);
        cudaEventElapsedTime(&tot, t_ev[0], t_ev[3]);
        t_times.forward_ms = ms[0];
        t_times.adjoint_ms = ms[1];
        t_times.other_ms = tot - ms[0] - ms[1];
        t_times.forward_launches = t_launch[0];
        t_times.adjoint_launches = t_launch[1];
        t_times.other_launches = t_launch[2];
    }
    if (status & ST_BAD_VELOCITY) return fail(FWI_ERR_INVALID_ARG, "velocity not finite and positive");
    if (status & ST_CFL) return fail(FWI_ERR_CFL, "v dt/dx above the 3-D stability limit %g", CFL_3D);
    if (status & ST_TIMEOUT) return fail(FWI_ERR_TIMEOUT, "a device wait timed out");
    if (status & ST_NONFINITE) return fail(FWI_ERR_UNSTABLE, "non-finite wavefield");
    t_err.clear();
    return FWI_OK;
}

fwi_status check_ws3(const Plan3 &pl, void *ws, size_t ws_bytes) { return check_ws_bytes(ws, ws_bytes, pl.total); }

// forward modelling (seis), illumination (illum) and / or the offset-Hessian
// diagonal (offh, op FWI_OP_OFFSET_HESSIAN) of all shots
fwi_status forward3(const fwi_grid *grid, const fwi_geometry *geom, const fwi_options *opts, int op,
                    const float *v, float *seis, float *illum, float *offh, void *ws, size_t ws_bytes,
                    cudaStream_t st)
{
    Plan3 pl;
    fwi_status s = make_plan3(grid, geom, opts, op, true, pl);
    if (s != FWI_OK) return s;
    if ((s = check_ws3(pl, ws, ws_bytes)) != FWI_OK) return s;
    begin_call(st);
    if ((s = setup3(pl, v, ws, st)) != FWI_OK) return s;
    float *acc_i = illum ? at<float>(ws, pl.acc_i) : nullptr;
    float *acc_h = offh && pl.hmax >= 0 ? at<float>(ws, pl.acc_h) : nullptr;
    const int utt = opts ? opts->illum_mode : 0;
    for (int s0 = 0; s0 < pl.ns_all; s0 += pl.G) {
        const int g = std::min(pl.G, pl.ns_all - s0);
        if ((s = upload_tables3(pl, geom, s0, g, ws, st)) != FWI_OK) return s;
        float *sg = seis ? seis + (size_t)s0 * pl.nt * pl.nrec : nullptr;
        if ((s = run_forward3(pl, geom, s0, g, ws, sg, acc_i, acc_h, utt, op == FWI_OP_FORWARD_SAVE, st)) != FWI_OK)
            return s;
    }
    prof_record(1, st);
    prof_record(2, st);
    if (illum) {
        const float iscale = utt == FWI_ILLUM_U2 ? pl.L.dt : 1.0f / (pl.L.dt * pl.L.dt * pl.L.dt);
        cudaError_t e = launch_finish_accum_n((long long)pl.L.nz * pl.L.ny * pl.L.nx, acc_i, 1, 1, iscale, illum, st,
                                              opts && opts->hess_v6 ? v : nullptr);
        if (e != cudaSuccess) return cuda_fail(e, "illumination output");
        t_launch[2]++;
    }
    if (acc_h) {
        cudaError_t e = launch_finish_accum_n((long long)pl.L.nz * pl.L.ny * pl.L.nx, acc_h, 1, pl.hmax + 1,
                                              pl.L.dt, offh, st, opts->hess_v6 ? v : nullptr);
        if (e != cudaSuccess) return cuda_fail(e, "offset-Hessian output");
        t_launch[2]++;
    }
    prof_record(3, st);
    return finish3(pl, ws, st);
}

fwi_status gradient3(const fwi_grid *grid, const fwi_geometry *geom, const fwi_options *opts, const float *v,
                     const float *d_obs, float *grad, float *grad_pre, double *misfit, float *illum, float *offh,
                     void *ws, size_t ws_bytes, cudaStream_t st)
{
    Plan3 pl;
    fwi_status s = make_plan3(grid, geom, opts, FWI_OP_GRADIENT, true, pl);
    if (s != FWI_OK) return s;
    if (!v || !grad || (!d_obs && geom->nrec > 0)) return fail(FWI_ERR_INVALID_ARG, "v, d_obs or grad is NULL");
    if (offh && opts->hmax < 0) return fail(FWI_ERR_INVALID_ARG, "offh requested with hmax < 0");
    if ((s = check_ws3(pl, ws, ws_bytes)) != FWI_OK) return s;
    cudaError_t e;
    begin_call(st);
    if ((s = setup3(pl, v, ws, st)) != FWI_OK) return s;
    float *acc_i = at<float>(ws, pl.acc_i), *syn = at<float>(ws, pl.syn);
    float *acc_h = pl.hmax >= 0 ? at<float>(ws, pl.acc_h) : nullptr;
    double *J = at<double>(ws, pl.scal, 0);
    for (int s0 = 0; s0 < pl.ns_all; s0 += pl.G) {
        const int g = std::min(pl.G, pl.ns_all - s0);
        if ((s = upload_tables3(pl, geom, s0, g, ws, st)) != FWI_OK) return s;
        if ((s = run_forward3(pl, geom, s0, g, ws, syn, acc_i, acc_h, opts->illum_mode, true, st)) != FWI_OK)
            return s;
        const long long nsamp = (long long)g * pl.nt * pl.nrec;
        if (nsamp > 0) {
            const float *dg = d_obs + (size_t)s0 * pl.nt * pl.nrec;
            if ((e = launch_residual_ols(syn, dg, nsamp, opts->misfit == FWI_MISFIT_OLS ? J : nullptr, st)) !=
                cudaSuccess)
                return cuda_fail(e, "residual kernel");
            t_launch[2]++;
            if (opts->misfit == FWI_MISFIT_TIME_INTEGRAL) {
                if ((e = launch_time_integral(syn, g, pl.nt, pl.nrec, pl.L.dt, J, st)) != cudaSuccess)
                    return cuda_fail(e, "time-integral kernel");
                t_launch[2]++;
            }
        }
        if ((s = run_backward3(pl, geom, s0, g, ws, syn, st)) != FWI_OK) return s;
    }
    prof_record(1, st); // groups interleave the loops: the phase split is not kept
    prof_record(2, st);
    if ((e = launch_fold_grad3d(pl.L, at<float>(ws, pl.acc_g), v, grad, st)) != cudaSuccess)
        return cuda_fail(e, "fold kernel");
    t_launch[2]++;
    const long long nphys = (long long)pl.L.nz * pl.L.ny * pl.L.nx;
    const float iscale = opts->illum_mode == FWI_ILLUM_U2 ? pl.L.dt : 1.0f / (pl.L.dt * pl.L.dt * pl.L.dt);
    float *ill_out = illum ? illum : acc_i; // in place when not requested
    const float *v6 = opts->hess_v6 ? v : nullptr;
    if ((e = launch_finish_accum_n(nphys, acc_i, 1, 1, iscale, ill_out, st, v6)) != cudaSuccess)
        return cuda_fail(e, "illumination output");
    t_launch[2]++;
    float *off_out = nullptr;
    if (acc_h) {
        off_out = offh ? offh : acc_h;
        if ((e = launch_finish_accum_n(nphys, acc_h, 1, pl.hmax + 1, pl.L.dt, off_out, st, v6)) != cudaSuccess)
            return cuda_fail(e, "offset-Hessian output");
        t_launch[2]++;
    }
    if (grad_pre) {
        if (opts->precond == FWI_PRECOND_NONE) {
            if ((e = cudaMemcpyAsync(grad_pre, grad, nphys * sizeof(float), cudaMemcpyDeviceToDevice, st)) !=
                cudaSuccess)
                return cuda_fail(e, "copy");
        } else {
            const bool ill = opts->precond == FWI_PRECOND_ILLUM;
            if ((e = launch_precond_n(nphys, grad, ill ? ill_out : off_out, ill ? 1 : 2, pl.hmax, opts->eps, grad_pre,
                                      at<unsigned>(ws, pl.scal, 12), st)) != cudaSuccess)
                return cuda_fail(e, "precondition kernel");
            t_launch[2] += 2;
        }
    }
    if (misfit && (e = cudaMemcpyAsync(misfit, J, sizeof(double), cudaMemcpyDeviceToDevice, st)) != cudaSuccess)
        return cuda_fail(e, "copy");
    prof_record(3, st);
    return finish3(pl, ws, st);
}

// fwi_adjoint_apply on a 3-D grid: J^T of adj_src after fwi_forward(save = 1)
// on the same workspace, from its snapshots (one group: all shots)
fwi_status adjoint_apply3(const fwi_grid *grid, const fwi_geometry *geom, const fwi_options *opts, const float *v,
                          const float *adj_src, float *grad, void *ws, size_t ws_bytes, cudaStream_t st)
{
    Plan3 pl;
    fwi_status s = make_plan3(grid, geom, opts, FWI_OP_FORWARD_SAVE, true, pl);
    if (s != FWI_OK) return s;
    if (!v || !grad || (!adj_src && geom->nrec > 0)) return fail(FWI_ERR_INVALID_ARG, "v, adj_src or grad is NULL");
    if ((s = check_ws3(pl, ws, ws_bytes)) != FWI_OK) return s;
    begin_call(st);
    prof_record(1, st);
    // c2 and the sponge factor again from v, the imaging sum cleared; the
    // snapshots stay
    if ((s = setup3(pl, v, ws, st)) != FWI_OK) return s;
    if ((s = upload_tables3(pl, geom, 0, pl.G, ws, st)) != FWI_OK) return s;
    if ((s = run_backward3(pl, geom, 0, pl.G, ws, adj_src, st)) != FWI_OK) return s;
    prof_record(2, st);
    cudaError_t e;
    if ((e = launch_fold_grad3d(pl.L, at<float>(ws, pl.acc_g), v, grad, st)) != cudaSuccess)
        return cuda_fail(e, "fold kernel");
    t_launch[2]++;
    prof_record(3, st);
    return finish3(pl, ws, st);
}

// Plans of a batch of models in one workspace: model k's parts start at
// base[k]. Every model is checked as in fwi_adjoint_gradient; the models
// share opts and nt.
// The receivers of a fixed spread as nrec sources without receivers (the
// receiver Green's functions), planned as an offset-Hessian pass, followed in
// the workspace by the sources' wavelets (shot 0's, replicated).
struct RecvPlan {
    Plan pl;
    fwi_geometry g2{};
    std::vector<int> src;
    fwi_options o2{};
    int hmax = 0;
    size_t wav_off = 0, total = 0;
};

// every shot records at the same cells (coords: the coordinates are read)
fwi_status check_fixed_spread(const fwi_geometry *ge)
{
    if (ge->nrec < 1) return fail(FWI_ERR_INVALID_ARG, "the receiver factor needs receivers");
    for (int s = 1; s < ge->nshots; ++s)
        if (std::memcmp(ge->rec, ge->rec + 3 * (size_t)s * ge->nrec, 3 * (size_t)ge->nrec * sizeof(int)) != 0)
            return fail(FWI_ERR_INVALID_ARG, "the receiver factor needs a fixed spread (shot %d records elsewhere)", s);
    return FWI_OK;
}

fwi_status make_recv_plan(const fwi_grid *g, const fwi_geometry *ge, const fwi_options *o, bool coords, RecvPlan &rp)
{
    fwi_status s;
    if ((s = check_grid(g)) != FWI_OK) return s;
    if ((s = check_geom(g, ge, coords)) != FWI_OK) return s;
    if ((s = check_opts(o, FWI_OP_RECEIVER_FACTOR)) != FWI_OK) return s;
    if (coords && (s = check_fixed_spread(ge)) != FWI_OK) return s;
    if (ge->nrec < 1) return fail(FWI_ERR_INVALID_ARG, "the receiver factor needs receivers");
    rp.hmax = o ? std::max(o->hmax, 0) : 0;
    rp.o2 = o ? *o : fwi_options{FWI_MISFIT_OLS, FWI_ILLUM_U2, 0, FWI_PRECOND_NONE, 1e-3f, FWI_CKPT_SPONGE,
                                 FWI_SNAP_F32, 0, 0, 0};
    rp.o2.hmax = rp.hmax;
    rp.o2.precond = FWI_PRECOND_NONE;
    rp.g2.nshots = ge->nrec;
    rp.g2.nrec = 0;
    rp.g2.rec = nullptr;
    rp.g2.wavelet = ge->wavelet; // replaced by the replicated wavelets at the call
    if (coords) {
        rp.src.assign(ge->rec, ge->rec + 3 * (size_t)ge->nrec);
        rp.g2.src = rp.src.data();
    }
    if ((s = make_plan(g, &rp.g2, &rp.o2, FWI_OP_OFFSET_HESSIAN, coords, rp.pl)) != FWI_OK) return s;
    rp.wav_off = align_up(rp.pl.total);
    rp.total = rp.wav_off + (size_t)ge->nrec * g->nt * sizeof(float);
    return FWI_OK;
}

// workspace of fwi_plessix_mulder_hessian: the illumination plan of all
// shots, then one illumination buffer
size_t pm_workspace(const Plan &all) { return align_up(all.total) + (size_t)all.L.nz * all.L.nx * sizeof(float); }

// options of a call that allows NULL ones: the defaults (OLS, u^2
// illumination, no offset Hessian, sponge checkpoints)
const fwi_options *or_defaults(const fwi_options *o, fwi_options &store)
{
    if (o) return o;
    store = fwi_options{FWI_MISFIT_OLS, FWI_ILLUM_U2, -1, FWI_PRECOND_NONE, 1e-3f, FWI_CKPT_SPONGE, FWI_SNAP_F32, 0, 0, 0};
    return &store;
}

fwi_status make_batch(int nm, const fwi_grid *grids, const fwi_geometry *geoms, const fwi_options *opts,
                      bool coords, std::vector<Plan> &pl, std::vector<size_t> &base, size_t &total)
{
    if (nm < 1 || nm > FWI_BATCH_MAX) return fail(FWI_ERR_INVALID_ARG, "nmodels=%d outside 1..%d", nm, FWI_BATCH_MAX);
    if (!grids || !geoms) return fail(FWI_ERR_INVALID_ARG, "grids or geoms is NULL");
    if (!opts) return fail(FWI_ERR_INVALID_ARG, "options are NULL");
    if (nm > 1 && opts->ckpt != FWI_CKPT_SPONGE)
        return fail(FWI_ERR_INVALID_ARG, "a batch of several models needs ckpt = FWI_CKPT_SPONGE");
    pl.assign(nm, Plan{});
    base.assign(nm, 0);
    total = 0;
    for (int k = 0; k < nm; ++k) {
        fwi_status s = make_plan(&grids[k], &geoms[k], opts, FWI_OP_GRADIENT, coords, pl[k]);
        if (s != FWI_OK) return fail(s, "model %d: %s", k, t_err.c_str());
        if (grids[k].nt != grids[0].nt)
            return fail(FWI_ERR_INVALID_ARG, "model %d has nt=%d, model 0 nt=%d: a batch shares nt", k, grids[k].nt,
                        grids[0].nt);
        base[k] = total;
        total = align_up(total + pl[k].total);
    }
    // a launch runs one kernel for all models: the tile variants and chunks
    // of the model with the most work (padded points x shots); the workspace
    // does not depend on the tiling
    int kmax = 0;
    for (int k = 1; k < nm; ++k)
        if ((long long)pl[k].L.nzp * pl[k].L.nxp * pl[k].ns > (long long)pl[kmax].L.nzp * pl[kmax].L.nxp * pl[kmax].ns)
            kmax = k;
    for (int k = 0; k < nm; ++k) {
        if (k == kmax) continue;
        const StepKind fk = pl[k].with_offh ? STEP_FWD_OFFH : STEP_FWD;
        pl[k].tf = make_tiling(pl[k].L, pl[k].ns, fk, pl[kmax].tf.variant, pl[kmax].tf.chunk, pl[k].hmax);
        pl[k].tb = make_tiling(pl[k].L, pl[k].ns, STEP_BWD, pl[kmax].tb.variant, pl[kmax].tb.chunk);
    }
    return FWI_OK;
}

// events 1 and 2 bracket the backward loop; for calls without one they
// coincide, and for calls without a forward loop event 1 is the start.
} // namespace

extern "C" {

int fwi_version(void) { return 100; }

const char *fwi_last_error(void) { return t_err.c_str(); }

fwi_status fwi_profile_enable(int on)
{
    t_prof = on != 0;
    return FWI_OK;
}

fwi_status fwi_profile_last(fwi_phase_times *out)
{
    if (!out) return fail(FWI_ERR_INVALID_ARG, "out is NULL");
    *out = t_times;
    return FWI_OK;
}

fwi_status fwi_workspace_bytes(const fwi_grid *grid, const fwi_geometry *geom, const fwi_options *opts,
                               int op, size_t *bytes)
{
    if (!bytes) return fail(FWI_ERR_INVALID_ARG, "bytes is NULL");
    if (op < FWI_OP_FORWARD || op > FWI_OP_PM_HESSIAN) return fail(FWI_ERR_INVALID_ARG, "op=%d unknown", op);
    if (op == FWI_OP_PM_HESSIAN) {
        Plan pl;
        fwi_options dflt;
        fwi_status s = make_plan(grid, geom, or_defaults(opts, dflt), FWI_OP_ILLUMINATION, false, pl);
        if (s != FWI_OK) return s;
        *bytes = pm_workspace(pl);
        t_err.clear();
        return FWI_OK;
    }
    if (grid && grid->ndim == 3 && op == FWI_OP_PRECONDITION) {
        fwi_status s3 = check_grid3(grid);
        if (s3 != FWI_OK) return s3;
        *bytes = ALIGN; // the status word and the maximum (as fwi_precondition uses them)
        t_err.clear();
        return FWI_OK;
    }
    if (grid && grid->ndim == 3) {
        Plan3 p3;
        fwi_status s3 = make_plan3(grid, geom, opts, op, false, p3);
        if (s3 != FWI_OK) return s3;
        *bytes = p3.total;
        t_err.clear();
        return FWI_OK;
    }
    if (op == FWI_OP_RECEIVER_FACTOR) {
        RecvPlan rp;
        fwi_status s = make_recv_plan(grid, geom, opts, false, rp);
        if (s != FWI_OK) return s;
        *bytes = rp.total;
        t_err.clear();
        return FWI_OK;
    }
    Plan pl;
    fwi_status s = make_plan(grid, geom, opts, op, false, pl);
    if (s != FWI_OK) return s;
    *bytes = pl.total;
    t_err.clear();
    return FWI_OK;
}

fwi_status fwi_forward(const fwi_grid *grid, const fwi_geometry *geom, const fwi_options *opts,
                       const float *v, float *seis, int save, void *ws, size_t ws_bytes, void *stream)
{
    Trace trace_("fwi_forward");
    if (grid && grid->ndim == 3) {
        if (!v || (!seis && geom && geom->nrec > 0)) return fail(FWI_ERR_INVALID_ARG, "v or seis is NULL");
        return forward3(grid, geom, opts, save ? FWI_OP_FORWARD_SAVE : FWI_OP_FORWARD, v, seis, nullptr, nullptr, ws,
                        ws_bytes, static_cast<cudaStream_t>(stream));
    }
    Plan pl;
    fwi_status s = make_plan(grid, geom, opts, save ? FWI_OP_FORWARD_SAVE : FWI_OP_FORWARD, true, pl);
    if (s != FWI_OK) return s;
    if (!v || (!seis && geom->nrec > 0)) return fail(FWI_ERR_INVALID_ARG, "v or seis is NULL");
    if ((s = check_ws(pl, ws, ws_bytes)) != FWI_OK) return s;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    begin_call(st);
    if ((s = setup(pl, geom, v, ws, st)) != FWI_OK) return s;
    if ((s = run_forward(pl, geom, ws, seis, save != 0, nullptr, nullptr, 0, st)) != FWI_OK) return s;
    prof_record(1, st);
    prof_record(2, st);
    prof_record(3, st);
    return finish(pl, ws, st);
}

fwi_status fwi_adjoint_apply(const fwi_grid *grid, const fwi_geometry *geom, const fwi_options *opts,
                             const float *v, const float *adj_src, float *grad, void *ws, size_t ws_bytes,
                             void *stream)
{
    Trace trace_("fwi_adjoint_apply");
    if (grid && grid->ndim == 3)
        return adjoint_apply3(grid, geom, opts, v, adj_src, grad, ws, ws_bytes, static_cast<cudaStream_t>(stream));
    Plan pl;
    fwi_status s = make_plan(grid, geom, opts, FWI_OP_FORWARD_SAVE, true, pl);
    if (s != FWI_OK) return s;
    if (!v || !grad || (!adj_src && geom->nrec > 0)) return fail(FWI_ERR_INVALID_ARG, "v, adj_src or grad is NULL");
    if ((s = check_ws(pl, ws, ws_bytes)) != FWI_OK) return s;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    begin_call(st);
    prof_record(1, st);
    cudaError_t e;
    if ((e = cudaMemsetAsync(at<char>(ws, pl.scal), 0, pl.scal.bytes, st)) != cudaSuccess) return cuda_fail(e, "memset");
    if ((e = cudaMemsetAsync(at<char>(ws, pl.sched), 0, pl.sched.bytes, st)) != cudaSuccess) return cuda_fail(e, "memset");
    if ((s = upload_tables(pl, geom, ws, st)) != FWI_OK) return s;
    if ((s = run_backward(pl, geom, ws, adj_src, st)) != FWI_OK) return s;
    prof_record(2, st);
    if ((e = launch_fold_grad(pl.L, at<float>(ws, pl.acc_g), 1, v, grad, st)) != cudaSuccess)
        return cuda_fail(e, "fold kernel");
    t_launch[2]++;
    prof_record(3, st);
    return finish(pl, ws, st);
}

fwi_status fwi_adjoint_gradient(const fwi_grid *grid, const fwi_geometry *geom, const fwi_options *opts,
                                const float *v, const float *d_obs, float *grad, float *grad_pre, double *misfit,
                                float *illum, float *offh, void *ws, size_t ws_bytes, void *stream)
{
    Trace trace_("fwi_adjoint_gradient");
    if (grid && grid->ndim == 3)
        return gradient3(grid, geom, opts, v, d_obs, grad, grad_pre, misfit, illum, offh, ws, ws_bytes,
                         static_cast<cudaStream_t>(stream));
    Plan pl;
    fwi_status s = make_plan(grid, geom, opts, FWI_OP_GRADIENT, true, pl);
    if (s != FWI_OK) return s;
    if (!v || !grad || (!d_obs && geom->nrec > 0)) return fail(FWI_ERR_INVALID_ARG, "v, d_obs or grad is NULL");
    if (offh && opts->hmax < 0) return fail(FWI_ERR_INVALID_ARG, "offh requested with hmax < 0");
    if ((s = check_ws(pl, ws, ws_bytes)) != FWI_OK) return s;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    GradientIO io{v, d_obs, grad, grad_pre, misfit, illum, offh};
    if ((s = gradient_models(1, &pl, &geom, opts, &ws, &io, st)) != FWI_OK) return s;
    return finish(pl, ws, st);
}

fwi_status fwi_illumination(const fwi_grid *grid, const fwi_geometry *geom, const fwi_options *opts,
                            const float *v, float *illum, void *ws, size_t ws_bytes, void *stream)
{
    Trace trace_("fwi_illumination");
    if (grid && grid->ndim == 3) {
        if (!v || !illum) return fail(FWI_ERR_INVALID_ARG, "v or illum is NULL");
        return forward3(grid, geom, opts, FWI_OP_ILLUMINATION, v, nullptr, illum, nullptr, ws, ws_bytes,
                        static_cast<cudaStream_t>(stream));
    }
    Plan pl;
    fwi_status s = make_plan(grid, geom, opts, FWI_OP_ILLUMINATION, true, pl);
    if (s != FWI_OK) return s;
    if (!v || !illum) return fail(FWI_ERR_INVALID_ARG, "v or illum is NULL");
    if ((s = check_ws(pl, ws, ws_bytes)) != FWI_OK) return s;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    begin_call(st);
    if ((s = setup(pl, geom, v, ws, st)) != FWI_OK) return s;
    float *acc_i = at<float>(ws, pl.acc_i);
    if ((s = run_forward(pl, geom, ws, nullptr, false, acc_i, nullptr, opts->illum_mode, st)) != FWI_OK) return s;
    prof_record(1, st);
    prof_record(2, st);
    const float iscale = opts->illum_mode == FWI_ILLUM_U2 ? pl.L.dt : 1.0f / (pl.L.dt * pl.L.dt * pl.L.dt);
    cudaError_t e;
    if ((e = launch_finish_accum(pl.L, acc_i, 1, 1, iscale, illum, st, opts->hess_v6 ? v : nullptr)) != cudaSuccess)
        return cuda_fail(e, "illumination output");
    t_launch[2]++;
    prof_record(3, st);
    return finish(pl, ws, st);
}

fwi_status fwi_offset_hessian_diag(const fwi_grid *grid, const fwi_geometry *geom, const fwi_options *opts,
                                   const float *v, float *offh, void *ws, size_t ws_bytes, void *stream)
{
    Trace trace_("fwi_offset_hessian_diag");
    if (grid && grid->ndim == 3) {
        if (!v || !offh) return fail(FWI_ERR_INVALID_ARG, "v or offh is NULL");
        return forward3(grid, geom, opts, FWI_OP_OFFSET_HESSIAN, v, nullptr, nullptr, offh, ws, ws_bytes,
                        static_cast<cudaStream_t>(stream));
    }
    Plan pl;
    fwi_status s = make_plan(grid, geom, opts, FWI_OP_OFFSET_HESSIAN, true, pl);
    if (s != FWI_OK) return s;
    if (!v || !offh) return fail(FWI_ERR_INVALID_ARG, "v or offh is NULL");
    if ((s = check_ws(pl, ws, ws_bytes)) != FWI_OK) return s;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    begin_call(st);
    if ((s = setup(pl, geom, v, ws, st)) != FWI_OK) return s;
    float *acc_h = at<float>(ws, pl.acc_h);
    if ((s = run_forward(pl, geom, ws, nullptr, false, nullptr, acc_h, 0, st)) != FWI_OK) return s;
    prof_record(1, st);
    prof_record(2, st);
    cudaError_t e;
    if ((e = launch_finish_accum(pl.L, acc_h, 1, pl.hmax + 1, pl.L.dt, offh, st, opts->hess_v6 ? v : nullptr)) !=
        cudaSuccess)
        return cuda_fail(e, "offset-Hessian output");
    t_launch[2]++;
    prof_record(3, st);
    return finish(pl, ws, st);
}

fwi_status fwi_precondition(const fwi_grid *grid, const float *grad, const float *scale, int kind, int hmax,
                            float eps, float *out, void *ws, size_t ws_bytes, void *stream)
{
    Trace trace_("fwi_precondition");
    // elementwise over the physical grid: in 3-D only the status word and
    // the maximum live in the workspace
    const bool three = grid && grid->ndim == 3;
    Plan pl;
    Plan3 p3;
    fwi_status s = three ? check_grid3(grid) : make_plan(grid, nullptr, nullptr, FWI_OP_PRECONDITION, false, pl);
    if (s != FWI_OK) return s;
    if (three) {
        p3.scal = Part{0, ALIGN};
        p3.total = ALIGN;
    }
    if (!grad || !scale || !out) return fail(FWI_ERR_INVALID_ARG, "grad, scale or out is NULL");
    if (kind != FWI_PRECOND_ILLUM && kind != FWI_PRECOND_OFFSET) return fail(FWI_ERR_INVALID_ARG, "kind=%d", kind);
    if (kind == FWI_PRECOND_OFFSET && (hmax < 0 || hmax > FWI_HMAX_LIMIT))
        return fail(FWI_ERR_INVALID_ARG, "hmax=%d outside 0..%d", hmax, FWI_HMAX_LIMIT);
    if (!(eps > 0.f)) return fail(FWI_ERR_INVALID_ARG, "eps must be > 0");
    if ((s = three ? check_ws3(p3, ws, ws_bytes) : check_ws(pl, ws, ws_bytes)) != FWI_OK) return s;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    begin_call(st);
    prof_record(1, st);
    prof_record(2, st);
    const Part &scal = three ? p3.scal : pl.scal;
    const long long nphys = three ? (long long)grid->nz * grid->ny * grid->nx : (long long)pl.L.nz * pl.L.nx;
    cudaError_t e;
    if ((e = cudaMemsetAsync(at<char>(ws, scal), 0, scal.bytes, st)) != cudaSuccess) return cuda_fail(e, "memset");
    if ((e = launch_precond_n(nphys, grad, scale, kind, hmax, eps, out, at<unsigned>(ws, scal, 12), st)) != cudaSuccess)
        return cuda_fail(e, "precondition kernel");
    t_launch[2] += 2;
    prof_record(3, st);
    return three ? finish3(p3, ws, st) : finish(pl, ws, st);
}

fwi_status fwi_misfit(const fwi_grid *grid, const fwi_geometry *geom, const fwi_options *opts, const float *v,
                      const float *d_obs, double *misfit, void *ws, size_t ws_bytes, void *stream)
{
    Trace trace_("fwi_misfit");
    Plan pl;
    fwi_status s = make_plan(grid, geom, opts, FWI_OP_MISFIT, true, pl);
    if (s != FWI_OK) return s;
    if (!v || !misfit || (!d_obs && geom->nrec > 0)) return fail(FWI_ERR_INVALID_ARG, "v, d_obs or misfit is NULL");
    if ((s = check_ws(pl, ws, ws_bytes)) != FWI_OK) return s;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    begin_call(st);
    if ((s = setup(pl, geom, v, ws, st)) != FWI_OK) return s;
    float *syn = at<float>(ws, pl.syn);
    if ((s = run_forward(pl, geom, ws, syn, false, nullptr, nullptr, 0, st)) != FWI_OK) return s;
    prof_record(1, st);
    cudaError_t e;
    double *J = at<double>(ws, pl.scal, 0);
    const long long nsamp = (long long)pl.ns * pl.nt * pl.nrec;
    const bool integral = opts && opts->misfit == FWI_MISFIT_TIME_INTEGRAL;
    if (nsamp > 0) {
        if ((e = launch_residual_ols(syn, d_obs, nsamp, integral ? nullptr : J, st)) != cudaSuccess)
            return cuda_fail(e, "residual kernel");
        t_launch[2]++;
        if (integral) {
            if ((e = launch_time_integral(syn, pl.ns, pl.nt, pl.nrec, pl.L.dt, J, st)) != cudaSuccess)
                return cuda_fail(e, "time-integral kernel");
            t_launch[2]++;
        }
    }
    if ((e = cudaMemcpyAsync(misfit, J, sizeof(double), cudaMemcpyDeviceToDevice, st)) != cudaSuccess)
        return cuda_fail(e, "copy");
    prof_record(2, st);
    prof_record(3, st);
    return finish(pl, ws, st);
}

fwi_status fwi_receiver_factor(const fwi_grid *grid, const fwi_geometry *geom, const fwi_options *opts, int kind,
                               const float *v, float *out, void *ws, size_t ws_bytes, void *stream)
{
    Trace trace_("fwi_receiver_factor");
    fwi_status s;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    if (kind == FWI_RECV_PLESSIX_MULDER) {
        if ((s = check_grid(grid)) != FWI_OK) return s;
        if ((s = check_geom(grid, geom, true)) != FWI_OK) return s;
        if ((s = check_fixed_spread(geom)) != FWI_OK) return s;
        if (!out) return fail(FWI_ERR_INVALID_ARG, "out is NULL");
        int xmin, xmax;
        float zr;
        spread_extent(geom->rec, geom->nrec, xmin, xmax, zr);
        cudaError_t e = launch_pm_factor(grid->nz, grid->nx, grid->dx, (float)xmin * grid->dx,
                                         (float)xmax * grid->dx, zr, out, st);
        if (e != cudaSuccess) return cuda_fail(e, "receiver-factor kernel");
        t_err.clear();
        return FWI_OK;
    }
    if (kind != FWI_RECV_GREEN) return fail(FWI_ERR_INVALID_ARG, "kind=%d unknown", kind);
    RecvPlan rp;
    if ((s = make_recv_plan(grid, geom, opts, true, rp)) != FWI_OK) return s;
    if (!v || !out) return fail(FWI_ERR_INVALID_ARG, "v or out is NULL");
    if ((s = check_ws_bytes(ws, ws_bytes, rp.total)) != FWI_OK) return s;
    const Plan &pl = rp.pl;
    begin_call(st);
    cudaError_t e;
    float *wav = reinterpret_cast<float *>(static_cast<char *>(ws) + rp.wav_off);
    if ((e = launch_replicate_row(geom->wavelet, grid->nt, geom->nrec, wav, st)) != cudaSuccess)
        return cuda_fail(e, "wavelet copy");
    t_launch[2]++;
    rp.g2.wavelet = wav;
    if ((s = setup(pl, &rp.g2, v, ws, st)) != FWI_OK) return s;
    float *acc_h = at<float>(ws, pl.acc_h);
    if ((s = run_forward(pl, &rp.g2, ws, nullptr, false, nullptr, acc_h, 0, st)) != FWI_OK) return s;
    prof_record(1, st);
    prof_record(2, st);
    if ((e = launch_finish_accum(pl.L, acc_h, 1, rp.hmax + 1, pl.L.dt, out, st)) != cudaSuccess)
        return cuda_fail(e, "receiver-factor output");
    t_launch[2]++;
    prof_record(3, st);
    return finish(pl, ws, st);
}

fwi_status fwi_plessix_mulder_hessian(const fwi_grid *grid, const fwi_geometry *geom, const fwi_options *opts,
                                      const float *v, float *out, void *ws, size_t ws_bytes, void *stream)
{
    Trace trace_("fwi_plessix_mulder_hessian");
    // the plan of all shots bounds every run's plan; the run's illumination
    // goes to a buffer after it
    fwi_options dflt;
    opts = or_defaults(opts, dflt);
    Plan all;
    fwi_status s = make_plan(grid, geom, opts, FWI_OP_ILLUMINATION, true, all);
    if (s != FWI_OK) return s;
    if (geom->nrec < 1) return fail(FWI_ERR_INVALID_ARG, "the Plessix-Mulder Hessian needs receivers");
    if (!v || !out) return fail(FWI_ERR_INVALID_ARG, "v or out is NULL");
    if ((s = check_ws_bytes(ws, ws_bytes, pm_workspace(all))) != FWI_OK) return s;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const int mode = opts->illum_mode;
    const float iscale = mode == FWI_ILLUM_U2 ? all.L.dt : 1.0f / (all.L.dt * all.L.dt * all.L.dt);
    float *tmp = reinterpret_cast<float *>(static_cast<char *>(ws) + align_up(all.total));
    const size_t nrec3 = 3 * (size_t)geom->nrec;
    begin_call(st);
    cudaError_t e;
    if ((e = cudaMemsetAsync(out, 0, (size_t)grid->nz * grid->nx * sizeof(float), st)) != cudaSuccess)
        return cuda_fail(e, "memset");
    Plan pr;
    for (int s0 = 0, run = 0; s0 < geom->nshots; ++run) {
        int s1 = s0 + 1;
        while (s1 < geom->nshots && std::memcmp(geom->rec + s1 * nrec3, geom->rec + s0 * nrec3, nrec3 * sizeof(int)) == 0)
            ++s1;
        fwi_geometry g{};
        g.nshots = s1 - s0;
        g.nrec = geom->nrec;
        g.src = geom->src + 3 * (size_t)s0;
        g.rec = geom->rec + s0 * nrec3;
        g.wavelet = geom->wavelet + (size_t)s0 * grid->nt;
        if ((s = make_plan(grid, &g, opts, FWI_OP_ILLUMINATION, true, pr)) != FWI_OK) return s;
        if (run == 0) {
            if ((s = setup(pr, &g, v, ws, st)) != FWI_OK) return s;
        } else {
            // c2 and the sponge factor stay (same v, same parts); the status
            // word keeps the earlier runs' bits
            if ((e = cudaMemsetAsync(at<char>(ws, pr.sched), 0, pr.sched.bytes, st)) != cudaSuccess)
                return cuda_fail(e, "memset");
            if ((s = upload_tables(pr, &g, ws, st)) != FWI_OK) return s;
            for (int b = 0; b < 2; ++b)
                if ((e = cudaMemsetAsync(at<char>(ws, pr.u[b]), 0, pr.u[b].bytes, st)) != cudaSuccess)
                    return cuda_fail(e, "memset");
        }
        float *acc_i = at<float>(ws, pr.acc_i);
        if ((e = cudaMemsetAsync(acc_i, 0, pr.acc_i.bytes, st)) != cudaSuccess) return cuda_fail(e, "memset");
        if ((s = run_forward(pr, &g, ws, nullptr, false, acc_i, nullptr, mode, st)) != FWI_OK) return s;
        if ((e = launch_finish_accum(pr.L, acc_i, 1, 1, iscale, tmp, st, opts->hess_v6 ? v : nullptr)) !=
            cudaSuccess)
            return cuda_fail(e, "illumination output");
        int xmin, xmax;
        float zr;
        spread_extent(g.rec, g.nrec, xmin, xmax, zr);
        if ((e = launch_pm_accumulate(grid->nz, grid->nx, grid->dx, (float)xmin * grid->dx, (float)xmax * grid->dx,
                                      zr, tmp, out, st)) != cudaSuccess)
            return cuda_fail(e, "Plessix-Mulder accumulation");
        t_launch[2] += 2;
        s0 = s1;
    }
    prof_record(1, st);
    prof_record(2, st);
    prof_record(3, st);
    return finish(pr, ws, st);
}

fwi_status fwi_precondition_receiver(const fwi_grid *grid, const float *grad, const float *scale, int kind,
                                     int hmax, const float *recv, int recv_planes, float eps, float *out, void *ws,
                                     size_t ws_bytes, void *stream)
{
    Trace trace_("fwi_precondition_receiver");
    Plan pl;
    fwi_status s = make_plan(grid, nullptr, nullptr, FWI_OP_PRECONDITION_RECEIVER, false, pl);
    if (s != FWI_OK) return s;
    if (!grad || !scale || !recv || !out) return fail(FWI_ERR_INVALID_ARG, "grad, scale, recv or out is NULL");
    if (kind != FWI_PRECOND_ILLUM && kind != FWI_PRECOND_OFFSET) return fail(FWI_ERR_INVALID_ARG, "kind=%d", kind);
    if (kind == FWI_PRECOND_OFFSET && (hmax < 0 || hmax > FWI_HMAX_LIMIT))
        return fail(FWI_ERR_INVALID_ARG, "hmax=%d outside 0..%d", hmax, FWI_HMAX_LIMIT);
    const int planes = kind == FWI_PRECOND_OFFSET ? hmax + 1 : 1;
    if (recv_planes != 1 && recv_planes < planes)
        return fail(FWI_ERR_INVALID_ARG, "recv_planes=%d: 1 or >= %d", recv_planes, planes);
    if (!(eps > 0.f)) return fail(FWI_ERR_INVALID_ARG, "eps must be > 0");
    if ((s = check_ws(pl, ws, ws_bytes)) != FWI_OK) return s;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    begin_call(st);
    prof_record(1, st);
    prof_record(2, st);
    cudaError_t e;
    const long long nphys = (long long)pl.L.nz * pl.L.nx;
    float *prod = at<float>(ws, pl.prod);
    if ((e = cudaMemsetAsync(at<char>(ws, pl.scal), 0, pl.scal.bytes, st)) != cudaSuccess) return cuda_fail(e, "memset");
    if ((e = launch_scale_product(nphys, planes, scale, recv, recv_planes, prod, st)) != cudaSuccess)
        return cuda_fail(e, "scale product");
    if ((e = launch_precond(pl.L, grad, prod, kind, hmax, eps, out, at<unsigned>(ws, pl.scal, 12), st)) != cudaSuccess)
        return cuda_fail(e, "precondition kernel");
    t_launch[2] += 3;
    prof_record(3, st);
    return finish(pl, ws, st);
}

fwi_status fwi_extended_born(const fwi_grid *grid, const fwi_geometry *geom, const fwi_options *opts, int hext,
                             const float *v, const float *dv_ext, float *dseis, void *ws, size_t ws_bytes, void *stream)
{
    Trace trace_("fwi_extended_born");
    Plan pl;
    fwi_status s = make_plan(grid, geom, opts, FWI_OP_EXT_BORN, true, pl);
    if (s != FWI_OK) return s;
    if (hext < 0 || hext > FWI_HEXT_LIMIT) return fail(FWI_ERR_INVALID_ARG, "hext=%d outside 0..%d", hext, FWI_HEXT_LIMIT);
    if (!v || !dv_ext || (!dseis && geom->nrec > 0)) return fail(FWI_ERR_INVALID_ARG, "v, dv_ext or dseis is NULL");
    if ((s = check_ws(pl, ws, ws_bytes)) != FWI_OK) return s;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    begin_call(st);
    if ((s = setup(pl, geom, v, ws, st)) != FWI_OK) return s;
    const int he = ext_kernel_he(hext);
    cudaError_t e;
    if ((e = cudaMemsetAsync(at<char>(ws, pl.dext), 0, pl.dext.bytes, st)) != cudaSuccess) return cuda_fail(e, "memset");
    if ((e = launch_prep_dext(pl.L, v, dv_ext, at<float>(ws, pl.c2), hext, he, at<float>(ws, pl.dext), st)) !=
        cudaSuccess)
        return cuda_fail(e, "prep kernel");
    t_launch[2]++;
    if ((s = run_born(pl, geom, ws, dseis, false, st, he)) != FWI_OK) return s;
    prof_record(1, st);
    prof_record(2, st);
    prof_record(3, st);
    return finish(pl, ws, st);
}

fwi_status fwi_extended_migration(const fwi_grid *grid, const fwi_geometry *geom, const fwi_options *opts, int hext,
                                  const float *v, const float *adj_src, float *image, void *ws, size_t ws_bytes,
                                  void *stream)
{
    Trace trace_("fwi_extended_migration");
    Plan pl;
    fwi_status s = make_plan(grid, geom, opts, FWI_OP_EXT_MIGRATION, true, pl);
    if (s != FWI_OK) return s;
    if (hext < 0 || hext > FWI_HEXT_LIMIT) return fail(FWI_ERR_INVALID_ARG, "hext=%d outside 0..%d", hext, FWI_HEXT_LIMIT);
    if (!v || !image || (!adj_src && geom->nrec > 0)) return fail(FWI_ERR_INVALID_ARG, "v, adj_src or image is NULL");
    if ((s = check_ws(pl, ws, ws_bytes)) != FWI_OK) return s;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    begin_call(st);
    if ((s = setup(pl, geom, v, ws, st)) != FWI_OK) return s;
    if ((s = run_forward(pl, geom, ws, nullptr, true, nullptr, nullptr, 0, st)) != FWI_OK) return s;
    prof_record(1, st);
    const int he = ext_kernel_he(hext);
    float *acc = at<float>(ws, pl.acc_ext);
    cudaError_t e;
    if ((e = cudaMemsetAsync(acc, 0, pl.acc_ext.bytes, st)) != cudaSuccess) return cuda_fail(e, "memset");
    const fwi_geometry *gp = geom;
    void *wp = ws;
    if ((s = run_backward_models(1, &pl, &gp, &wp, &adj_src, st, -1, 1, nullptr, nullptr, he, acc)) != FWI_OK)
        return s;
    prof_record(2, st);
    if ((e = launch_fold_ext(pl.L, acc, he, hext, v, image, st)) != cudaSuccess) return cuda_fail(e, "fold kernel");
    t_launch[2]++;
    prof_record(3, st);
    return finish(pl, ws, st);
}

fwi_status fwi_selftest_wait(unsigned limit_us, void *ws, size_t ws_bytes, void *stream)
{
    if (limit_us < 1 || limit_us > 10000000u) return fail(FWI_ERR_INVALID_ARG, "limit_us=%u outside 1..10000000", limit_us);
    fwi_status s;
    if ((s = check_ws_bytes(ws, ws_bytes, 256)) != FWI_OK) return s;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    int *status = static_cast<int *>(ws);
    int h = 0;
    cudaError_t e;
    if ((e = cudaMemsetAsync(status, 0, sizeof(int), st)) != cudaSuccess) return cuda_fail(e, "memset");
    if ((e = launch_wait_selftest((uint64_t)limit_us * 1000ull, status, st)) != cudaSuccess)
        return cuda_fail(e, "self-test kernel");
    if ((e = cudaMemcpyAsync(&h, status, sizeof(int), cudaMemcpyDeviceToHost, st)) != cudaSuccess ||
        (e = cudaStreamSynchronize(st)) != cudaSuccess)
        return cuda_fail(e, "status read-back");
    if (h & ST_TIMEOUT) return fail(FWI_ERR_TIMEOUT, "the self-test wait gave up after %u us, as designed", limit_us);
    return fail(FWI_ERR_CUDA, "the self-test wait did not report its timeout (status %d)", h);
}

// dc2 = 2 c2 dv / v of a Born call on its padded grid (after setup's c2)
fwi_status prep_dc2(const Plan &pl, const float *v, const float *dv, void *ws, cudaStream_t st)
{
    cudaError_t e;
    if ((e = cudaMemsetAsync(at<char>(ws, pl.dc2), 0, pl.dc2.bytes, st)) != cudaSuccess) return cuda_fail(e, "memset");
    if ((e = launch_prep_dc2(pl.L, v, dv, at<float>(ws, pl.c2), at<float>(ws, pl.dc2), st)) != cudaSuccess)
        return cuda_fail(e, "prep kernel");
    t_launch[2]++;
    return FWI_OK;
}

fwi_status fwi_born(const fwi_grid *grid, const fwi_geometry *geom, const fwi_options *opts, const float *v,
                    const float *dv, float *dseis, void *ws, size_t ws_bytes, void *stream)
{
    Trace trace_("fwi_born");
    Plan pl;
    fwi_status s = make_plan(grid, geom, opts, FWI_OP_BORN, true, pl);
    if (s != FWI_OK) return s;
    if (!v || !dv || (!dseis && geom->nrec > 0)) return fail(FWI_ERR_INVALID_ARG, "v, dv or dseis is NULL");
    if ((s = check_ws(pl, ws, ws_bytes)) != FWI_OK) return s;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    begin_call(st);
    if ((s = setup(pl, geom, v, ws, st)) != FWI_OK) return s;
    if ((s = prep_dc2(pl, v, dv, ws, st)) != FWI_OK) return s;
    if ((s = run_born(pl, geom, ws, dseis, false, st)) != FWI_OK) return s;
    prof_record(1, st);
    prof_record(2, st);
    prof_record(3, st);
    return finish(pl, ws, st);
}

fwi_status fwi_gauss_newton_hvp(const fwi_grid *grid, const fwi_geometry *geom, const fwi_options *opts,
                                const float *v, const float *dv, float *hv, void *ws, size_t ws_bytes, void *stream)
{
    Trace trace_("fwi_gauss_newton_hvp");
    Plan pl;
    fwi_status s = make_plan(grid, geom, opts, FWI_OP_GN_HVP, true, pl);
    if (s != FWI_OK) return s;
    if (!v || !dv || !hv) return fail(FWI_ERR_INVALID_ARG, "v, dv or hv is NULL");
    if ((s = check_ws(pl, ws, ws_bytes)) != FWI_OK) return s;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    begin_call(st);
    if ((s = setup(pl, geom, v, ws, st)) != FWI_OK) return s;
    cudaError_t e;
    if ((s = prep_dc2(pl, v, dv, ws, st)) != FWI_OK) return s;
    float *dseis = at<float>(ws, pl.syn);
    if ((s = run_born(pl, geom, ws, dseis, true, st)) != FWI_OK) return s;
    prof_record(1, st);
    if (opts && opts->misfit == FWI_MISFIT_TIME_INTEGRAL && (long long)pl.ns * pl.nrec > 0) {
        // W^T W = C^T C of Eq. 2 on the Born traces (the misfit of the Born
        // traces goes to the call's scratch word)
        if ((e = launch_time_integral(dseis, pl.ns, pl.nt, pl.nrec, pl.L.dt, at<double>(ws, pl.scal, 0), st)) !=
            cudaSuccess)
            return cuda_fail(e, "time-integral kernel");
        t_launch[2]++;
    }
    if ((s = run_backward(pl, geom, ws, dseis, st)) != FWI_OK) return s;
    prof_record(2, st);
    if ((e = launch_fold_grad(pl.L, at<float>(ws, pl.acc_g), 1, v, hv, st)) != cudaSuccess)
        return cuda_fail(e, "fold kernel");
    t_launch[2]++;
    prof_record(3, st);
    return finish(pl, ws, st);
}

// fwi_autotune of a 3-D gradient: every compiled variant of the forward and
// backward steps timed on a few levels of the first shot group (the second
// of two passes), the fastest kept for the shape
fwi_status autotune3(const fwi_grid *grid, const fwi_geometry *geom, const fwi_options *opts, const float *v,
                     void *ws, size_t ws_bytes, cudaStream_t st, int *choice)
{
    Plan3 pl;
    fwi_status s = make_plan3(grid, geom, opts, FWI_OP_GRADIENT, true, pl);
    if (s != FWI_OK) return s;
    if (!v) return fail(FWI_ERR_INVALID_ARG, "v is NULL");
    if ((s = check_ws3(pl, ws, ws_bytes)) != FWI_OK) return s;
    const bool prof = t_prof;
    t_prof = false;
    struct Ev {
        cudaEvent_t a = nullptr, b = nullptr;
        ~Ev()
        {
            if (a) cudaEventDestroy(a);
            if (b) cudaEventDestroy(b);
        }
    } ev;
    cudaError_t e;
    if ((e = cudaEventCreate(&ev.a)) != cudaSuccess || (e = cudaEventCreate(&ev.b)) != cudaSuccess)
        return cuda_fail(e, "cudaEventCreate");
    if ((s = setup3(pl, v, ws, st)) != FWI_OK) return s;
    if ((s = upload_tables3(pl, geom, 0, pl.G, ws, st)) != FWI_OK) return s;
    const int nlev = std::min(6, pl.nt - 1);
    int best[2] = {0, 0};
    for (int b = 0; b < 2 && s == FWI_OK; ++b) {
        float best_ms = 1e30f;
        for (int vi = 0; vi < step3_variants(b != 0) && s == FWI_OK; ++vi) {
            Plan3 p = pl;
            if (b == 0) {
                p.vf = vi;
                p.tf = make_tiling3(p.L, p.G, false, vi);
            } else {
                p.vb = vi;
                p.tb = make_tiling3(p.L, p.G, true, vi);
            }
            float ms = 0.f;
            for (int rep = 0; rep < 2 && s == FWI_OK; ++rep) { // first pass warms up
                s = b == 0 ? run_forward3(p, geom, 0, p.G, ws, nullptr, nullptr, nullptr, 0, false, st, 1,
                                          1 + nlev, ev.a, ev.b)
                           : time_backward3(p, geom, ws, nlev, st, ev.a, ev.b);
                if (s == FWI_OK && (e = cudaEventSynchronize(ev.b)) != cudaSuccess) s = cuda_fail(e, "sync");
                if (s == FWI_OK) cudaEventElapsedTime(&ms, ev.a, ev.b);
            }
            if (s == FWI_OK && ms < best_ms) {
                best_ms = ms;
                best[b] = vi;
            }
        }
        if (s == FWI_OK) step3_tuned_store(pl.L, pl.G, b != 0, best[b], 0);
    }
    t_prof = prof;
    if (s != FWI_OK) return s;
    if ((e = cudaStreamSynchronize(st)) != cudaSuccess) return cuda_fail(e, "synchronize");
    if (choice) {
        choice[0] = best[0];
        choice[1] = make_tiling3(pl.L, pl.G, false, best[0]).nseg;
        choice[2] = best[1];
        choice[3] = make_tiling3(pl.L, pl.G, true, best[1]).nseg;
    }
    t_err.clear();
    return FWI_OK;
}

fwi_status fwi_autotune(const fwi_grid *grid, const fwi_geometry *geom, const fwi_options *opts, const float *v,
                        void *ws, size_t ws_bytes, void *stream, int *choice)
{
    Trace trace_("fwi_autotune");
    if (grid && grid->ndim == 3)
        return autotune3(grid, geom, opts, v, ws, ws_bytes, static_cast<cudaStream_t>(stream), choice);
    Plan pl;
    fwi_status s = make_plan(grid, geom, opts, FWI_OP_GRADIENT, true, pl);
    if (s != FWI_OK) return s;
    if (!v) return fail(FWI_ERR_INVALID_ARG, "v is NULL");
    if ((s = check_ws(pl, ws, ws_bytes)) != FWI_OK) return s;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const bool prof = t_prof;
    t_prof = false;
    struct Ev {
        cudaEvent_t a = nullptr, b = nullptr;
        ~Ev()
        {
            if (a) cudaEventDestroy(a);
            if (b) cudaEventDestroy(b);
        }
    } ev;
    cudaError_t e;
    if ((e = cudaEventCreate(&ev.a)) != cudaSuccess || (e = cudaEventCreate(&ev.b)) != cudaSuccess)
        return cuda_fail(e, "cudaEventCreate");
    if ((s = setup(pl, geom, v, ws, st)) != FWI_OK) return s;
    const int nt = pl.nt;
    const int nlev = std::min(8, nt - 1), n0 = std::max(0, (nt - nlev) / 2);
    float *acc_i = at<float>(ws, pl.acc_i), *acc_h = pl.with_offh ? at<float>(ws, pl.acc_h) : nullptr;
    float *syn = at<float>(ws, pl.syn);
    const StepKind fk = pl.with_offh ? STEP_FWD_OFFH : STEP_FWD;
    const StepKind kinds[2] = {fk, STEP_BWD};
    int best[2][2] = {{0, 0}, {0, 0}};
    for (int kk = 0; kk < 2; ++kk) {
        const StepKind kind = kinds[kk];
        const int *chunks = nullptr;
        const int nc = step_chunks(kind, &chunks), nv = step_variants(kind);
        float best_ms = 1e30f;
        for (int vi = 0; vi < nv; ++vi)
            for (int ci = 0; ci < nc; ++ci) {
                if (!step_variant_valid(kind, vi, pl.hmax)) continue;
                Plan p = pl;
                if (kk == 0)
                    p.tf = make_tiling(p.L, p.ns, kind, vi, chunks[ci], pl.hmax);
                else
                    p.tb = make_tiling(p.L, p.ns, kind, vi, chunks[ci]);
                if ((s = upload_tables(p, geom, ws, st)) != FWI_OK) break;
                float ms = 0.f;
                for (int rep = 0; rep < 2 && s == FWI_OK; ++rep) { // first pass warms up
                    if ((e = cudaMemsetAsync(at<char>(ws, p.sched), 0, p.sched.bytes, st)) != cudaSuccess) {
                        s = cuda_fail(e, "memset");
                        break;
                    }
                    const fwi_geometry *gp = geom;
                    void *wp = ws;
                    if (kk == 0) {
                        float *sp = syn;
                        s = run_forward_models(1, &p, &gp, &wp, &sp, true, &acc_i, &acc_h, opts->illum_mode, st, n0,
                                               n0 + nlev, ev.a, ev.b);
                    } else {
                        const float *ap = syn;
                        // levels m in [1, nt-1] (the adjoint source has nt levels)
                        s = run_backward_models(1, &p, &gp, &wp, &ap, st, std::min(nt - 1, n0 + nlev),
                                                std::max(1, n0 + 1), ev.a, ev.b);
                    }
                    if (s == FWI_OK && (e = cudaEventSynchronize(ev.b)) != cudaSuccess) s = cuda_fail(e, "sync");
                    if (s == FWI_OK) cudaEventElapsedTime(&ms, ev.a, ev.b);
                }
                if (s != FWI_OK) break;
                if (ms < best_ms) {
                    best_ms = ms;
                    best[kk][0] = vi;
                    best[kk][1] = chunks[ci];
                }
            }
        if (s != FWI_OK) break;
        step_tuned_store(kind, pl.L, pl.ns, best[kk][0], best[kk][1]);
    }
    t_prof = prof;
    if (s != FWI_OK) return s;
    // status words written while timing (the timing fields are not a
    // gradient) are cleared by the next call's set-up
    if ((e = cudaStreamSynchronize(st)) != cudaSuccess) return cuda_fail(e, "synchronize");
    if (choice) {
        choice[0] = best[0][0];
        choice[1] = best[0][1];
        choice[2] = best[1][0];
        choice[3] = best[1][1];
    }
    t_err.clear();
    return FWI_OK;
}

fwi_status fwi_autotune_set(const fwi_grid *grid, const fwi_geometry *geom, const fwi_options *opts,
                            const int *choice)
{
    if (!choice) return fail(FWI_ERR_INVALID_ARG, "choice is NULL");
    if (grid && grid->ndim == 3) {
        Plan3 p3;
        fwi_status s3 = make_plan3(grid, geom, opts, FWI_OP_GRADIENT, false, p3);
        if (s3 != FWI_OK) return s3;
        if (choice[0] < 0 || choice[0] >= step3_variants(false) || choice[2] < 0 || choice[2] >= step3_variants(true))
            return fail(FWI_ERR_INVALID_ARG, "variant outside the compiled ones (%d forward, %d backward)",
                        step3_variants(false), step3_variants(true));
        if (choice[1] < 0 || choice[3] < 0)
            return fail(FWI_ERR_INVALID_ARG, "3-D z-segments must be >= 0 (0: chosen per launch shape)");
        step3_tuned_store(p3.L, p3.G, false, choice[0], choice[1]);
        step3_tuned_store(p3.L, p3.G, true, choice[2], choice[3]);
        t_err.clear();
        return FWI_OK;
    }
    Plan pl;
    fwi_status s = make_plan(grid, geom, opts, FWI_OP_GRADIENT, false, pl);
    if (s != FWI_OK) return s;
    const StepKind fk = pl.with_offh ? STEP_FWD_OFFH : STEP_FWD;
    if (!step_variant_valid(fk, choice[0], pl.hmax) || !step_variant_valid(STEP_BWD, choice[2], pl.hmax))
        return fail(FWI_ERR_INVALID_ARG, "variant outside the compiled ones (%d forward, %d backward) or not "
                    "covering hmax=%d", step_variants(fk), step_variants(STEP_BWD), pl.hmax);
    if (choice[1] < 1 || choice[3] < 1) return fail(FWI_ERR_INVALID_ARG, "chunk must be >= 1");
    step_tuned_store(fk, pl.L, pl.ns, choice[0], choice[1]);
    step_tuned_store(STEP_BWD, pl.L, pl.ns, choice[2], choice[3]);
    t_err.clear();
    return FWI_OK;
}

fwi_status fwi_autotune_reset(void)
{
    step_tuned_clear();
    step3_tuned_clear();
    return FWI_OK;
}

fwi_status fwi_batch_workspace_bytes(int nmodels, const fwi_grid *grids, const fwi_geometry *geoms,
                                     const fwi_options *opts, size_t *bytes)
{
    if (!bytes) return fail(FWI_ERR_INVALID_ARG, "bytes is NULL");
    std::vector<Plan> pl;
    std::vector<size_t> base;
    size_t total = 0;
    fwi_status s = make_batch(nmodels, grids, geoms, opts, false, pl, base, total);
    if (s != FWI_OK) return s;
    *bytes = total;
    t_err.clear();
    return FWI_OK;
}

} // extern "C"

namespace {
// Checked arguments of a gradient over a batch of models.
struct BatchCall {
    std::vector<Plan> pl;
    std::vector<GradientIO> io;
    std::vector<void *> wk;
    std::vector<const fwi_geometry *> gp;
};

fwi_status batch_prepare(int nmodels, const fwi_grid *grids, const fwi_geometry *geoms, const fwi_options *opts,
                         const float *const *v, const float *const *d_obs, float *const *grad,
                         float *const *grad_pre, double *misfit, float *const *illum, float *const *offh, void *ws,
                         size_t ws_bytes, BatchCall &bc)
{
    std::vector<size_t> base;
    size_t total = 0;
    fwi_status s = make_batch(nmodels, grids, geoms, opts, true, bc.pl, base, total);
    if (s != FWI_OK) return s;
    if (!v || !grad || !d_obs) return fail(FWI_ERR_INVALID_ARG, "v, d_obs or grad is NULL");
    std::vector<GradientIO> &io = bc.io;
    std::vector<void *> &wk = bc.wk;
    io.assign(nmodels, GradientIO{});
    wk.assign(nmodels, nullptr);
    for (int k = 0; k < nmodels; ++k) {
        if (!v[k] || !grad[k] || (!d_obs[k] && geoms[k].nrec > 0))
            return fail(FWI_ERR_INVALID_ARG, "model %d: v, d_obs or grad is NULL", k);
        io[k] = GradientIO{v[k], d_obs[k], grad[k], grad_pre ? grad_pre[k] : nullptr,
                           misfit ? misfit + k : nullptr, illum ? illum[k] : nullptr, offh ? offh[k] : nullptr};
        if (io[k].offh && opts->hmax < 0) return fail(FWI_ERR_INVALID_ARG, "offh requested with hmax < 0");
        wk[k] = static_cast<char *>(ws) + base[k];
    }
    if ((s = check_ws_bytes(ws, ws_bytes, total)) != FWI_OK) return s;
    bc.gp.assign(nmodels, nullptr);
    for (int k = 0; k < nmodels; ++k) bc.gp[k] = &geoms[k];
    return FWI_OK;
}
} // namespace

// A recorded gradient: the device work of one gradient call as a CUDA graph,
// bound to the buffers it was recorded with.
struct fwi_exec_s {
    std::vector<Plan> pl;
    std::vector<void *> wk;
    cudaEvent_t input_ev = nullptr; // the misfit waits on it (fwi_exec_input_ready)
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    bool prof = false;
    int launches[3] = {0, 0, 0};
};

extern "C" {

fwi_status fwi_batch_gradient(int nmodels, const fwi_grid *grids, const fwi_geometry *geoms,
                              const fwi_options *opts, const float *const *v, const float *const *d_obs,
                              float *const *grad, float *const *grad_pre, double *misfit, float *const *illum,
                              float *const *offh, void *ws, size_t ws_bytes, void *stream)
{
    Trace trace_("fwi_batch_gradient");
    BatchCall bc;
    fwi_status s = batch_prepare(nmodels, grids, geoms, opts, v, d_obs, grad, grad_pre, misfit, illum, offh, ws,
                                 ws_bytes, bc);
    if (s != FWI_OK) return s;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    if ((s = gradient_models(nmodels, bc.pl.data(), bc.gp.data(), opts, bc.wk.data(), bc.io.data(), st)) != FWI_OK)
        return s;
    return finish_models(nmodels, bc.pl.data(), bc.wk.data(), st);
}

fwi_status fwi_exec_gradient_create(int nmodels, const fwi_grid *grids, const fwi_geometry *geoms,
                                    const fwi_options *opts, const float *const *v, const float *const *d_obs,
                                    float *const *grad, float *const *grad_pre, double *misfit,
                                    float *const *illum, float *const *offh, void *ws, size_t ws_bytes,
                                    void *stream, fwi_exec **out)
{
    Trace trace_("fwi_exec_gradient_create");
    if (!out) return fail(FWI_ERR_INVALID_ARG, "out is NULL");
    *out = nullptr;
    if (!stream) return fail(FWI_ERR_INVALID_ARG, "recording a graph needs a stream other than the default stream");
    BatchCall bc;
    fwi_status s = batch_prepare(nmodels, grids, geoms, opts, v, d_obs, grad, grad_pre, misfit, illum, offh, ws,
                                 ws_bytes, bc);
    if (s != FWI_OK) return s;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    // the geometry tables do not change between runs: uploaded once, here
    for (int k = 0; k < nmodels; ++k)
        if ((s = upload_tables(bc.pl[k], bc.gp[k], bc.wk[k], st)) != FWI_OK) return s;
    cudaError_t e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return cuda_fail(e, "synchronize");
    fwi_exec *ex = new fwi_exec_s;
    ex->pl = bc.pl;
    ex->wk = bc.wk;
    ex->prof = t_prof;
    if ((e = cudaEventCreateWithFlags(&ex->input_ev, cudaEventDisableTiming)) != cudaSuccess) {
        delete ex;
        return cuda_fail(e, "cudaEventCreate");
    }
    if ((e = cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal)) != cudaSuccess) {
        cudaEventDestroy(ex->input_ev);
        delete ex;
        return cuda_fail(e, "cudaStreamBeginCapture");
    }
    t_capturing = true;
    s = gradient_models(nmodels, bc.pl.data(), bc.gp.data(), opts, bc.wk.data(), bc.io.data(), st, false,
                        ex->input_ev);
    t_capturing = false;
    e = cudaStreamEndCapture(st, &ex->graph);
    if (s == FWI_OK && e != cudaSuccess) s = cuda_fail(e, "cudaStreamEndCapture");
    if (s == FWI_OK && (e = cudaGraphInstantiate(&ex->exec, ex->graph, 0)) != cudaSuccess)
        s = cuda_fail(e, "cudaGraphInstantiate");
    if (s != FWI_OK) {
        if (ex->graph) cudaGraphDestroy(ex->graph);
        cudaEventDestroy(ex->input_ev);
        delete ex;
        return s;
    }
    for (int i = 0; i < 3; ++i) ex->launches[i] = t_launch[i];
    *out = ex;
    t_err.clear();
    return FWI_OK;
}

fwi_status fwi_exec_input_ready(fwi_exec *ex, void *stream)
{
    if (!ex || !ex->exec) return fail(FWI_ERR_INVALID_ARG, "exec is NULL");
    cudaError_t e = cudaEventRecord(ex->input_ev, static_cast<cudaStream_t>(stream));
    if (e != cudaSuccess) return cuda_fail(e, "cudaEventRecord");
    t_err.clear();
    return FWI_OK;
}

fwi_status fwi_exec_run(fwi_exec *ex, void *stream)
{
    Trace trace_("fwi_exec_run");
    if (!ex || !ex->exec) return fail(FWI_ERR_INVALID_ARG, "exec is NULL");
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    t_ev_recorded = ex->prof && t_prof && t_ev[0];
    cudaError_t e = cudaGraphLaunch(ex->exec, st);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGraphLaunch");
    for (int i = 0; i < 3; ++i) t_launch[i] = ex->launches[i];
    return finish_models((int)ex->pl.size(), ex->pl.data(), ex->wk.data(), st);
}

fwi_status fwi_exec_destroy(fwi_exec *ex)
{
    if (!ex) return FWI_OK;
    if (ex->exec) cudaGraphExecDestroy(ex->exec);
    if (ex->graph) cudaGraphDestroy(ex->graph);
    if (ex->input_ev) cudaEventDestroy(ex->input_ev);
    delete ex;
    return FWI_OK;
}

} // extern "C"

// --------------------------------------------------------------------------
// Forward modelling without a caller workspace.
//
// Some callers cannot allocate device memory: code that runs where cudaMalloc
// is not allowed or not wanted (inside a region that must not synchronise the
// device, a host framework that owns all device memory through its own pool,
// or a plugin that is handed only input and output buffers). For them
// fwi_forward_noalloc() runs the same forward modelling as fwi_forward(save=0)
// in a scratch array that the library itself holds: a file-scope __device__
// array of FWI_NOALLOC_SCRATCH_BYTES, present on every GPU that loads this
// part of the library until the process exits. The entry point calls no
// cudaMalloc, cudaFree or other allocating routine on the device.
namespace {

static __device__ __align__(256) unsigned char g_noalloc_scratch[FWI_NOALLOC_SCRATCH_BYTES];

constexpr int NOALLOC_MAX_DEVICES = 64;
std::mutex g_noalloc_mu;
struct NoallocSlot {
    void *ptr;               // device address of the scratch array
    unsigned long long ctx;  // context it was looked up in
};
NoallocSlot g_noalloc[NOALLOC_MAX_DEVICES] = {};

// Unique id of the calling thread's current context; false when no context
// is current yet (or the driver entry points are unavailable).
bool current_context_id(unsigned long long &id)
{
    static PFN_cuCtxGetCurrent_v4000 get_current = nullptr;
    static PFN_cuCtxGetId_v12000 get_id = nullptr;
    static std::once_flag once;
    std::call_once(once, [] {
        void *fn = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &fn, 4000, cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            get_current = reinterpret_cast<PFN_cuCtxGetCurrent_v4000>(fn);
        fn = nullptr;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetId", &fn, 12000, cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            get_id = reinterpret_cast<PFN_cuCtxGetId_v12000>(fn);
        cudaGetLastError();
    });
    CUcontext ctx = nullptr;
    if (!get_current || !get_id || get_current(&ctx) != CUDA_SUCCESS || !ctx) return false;
    return get_id(ctx, &id) == CUDA_SUCCESS;
}

// Device address of the scratch array on the current device (host code sees
// only a host-side stand-in under its name). Looked up once per device and
// context: after a device reset the new context may place the array
// elsewhere, so a changed context id triggers a new lookup.
fwi_status noalloc_scratch(void **ptr)
{
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGetDevice");
    if (dev < 0 || dev >= NOALLOC_MAX_DEVICES) return fail(FWI_ERR_INVALID_ARG, "device %d out of range", dev);
    unsigned long long id = 0;
    const bool have_id = current_context_id(id);
    std::lock_guard<std::mutex> lock(g_noalloc_mu);
    NoallocSlot &sl = g_noalloc[dev];
    if (!sl.ptr || !have_id || sl.ctx != id) {
        void *p = nullptr;
        e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess || !p) return cuda_fail(e, "cudaGetSymbolAddress of the library scratch");
        if (!have_id && !current_context_id(id)) id = 0; // the lookup made the context current
        sl.ptr = p;
        sl.ctx = id;
    }
    *ptr = sl.ptr;
    return FWI_OK;
}

} // namespace

extern "C" fwi_status fwi_forward_noalloc(const fwi_grid *grid, const fwi_geometry *geom, const float *v,
                                          float *seis, void *stream)
{
    Trace trace_("fwi_forward_noalloc");
    Plan pl;
    fwi_status s = make_plan(grid, geom, nullptr, FWI_OP_FORWARD, true, pl);
    if (s != FWI_OK) return s;
    if (!v || (!seis && geom->nrec > 0)) return fail(FWI_ERR_INVALID_ARG, "v or seis is NULL");
    if (pl.total > (size_t)FWI_NOALLOC_SCRATCH_BYTES)
        return fail(FWI_ERR_NOMEM,
                    "this problem needs %zu bytes of scratch; fwi_forward_noalloc holds %zu "
                    "(use fwi_forward with a workspace of fwi_workspace_bytes(FWI_OP_FORWARD))",
                    pl.total, (size_t)FWI_NOALLOC_SCRATCH_BYTES);
    void *ws = nullptr;
    if ((s = noalloc_scratch(&ws)) != FWI_OK) return s;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    begin_call(st);
    // set-up clears everything that must start at zero (status, c2 ghost
    // frame, both wavefields): the scratch keeps the previous call's contents
    if ((s = setup(pl, geom, v, ws, st)) != FWI_OK) return s;
    if ((s = run_forward(pl, geom, ws, seis, false, nullptr, nullptr, 0, st)) != FWI_OK) return s;
    prof_record(1, st);
    prof_record(2, st);
    prof_record(3, st);
    return finish(pl, ws, st);
}
