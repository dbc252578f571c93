// fwi_step2d.cu -- time-step kernels of the 2-D FWI gradient (sm_103a).
//
// Forward step (one launch per time level n, all shots):
//   (1 + eta dt) u^{n+1} = 2 u^n - (1 - eta dt) u^{n-1} + c2 (Lhat u^n + f_s(t_n) delta_s)
// with c2 = (v dt/dx)^2 and Lhat the 8th-order Laplacian without 1/dx^2: the
// leapfrog discretisation of the constant-density acoustic equation of Sec. 2
// with an absorbing sponge u_tt + 2 eta u_t. Fused into the same pass over the
// tile: receiver extraction d^n = R u^n [Sec. 2], the shot illumination of
// Eq. 1 (sum u^2, or the u_tt^2 form), the offset-Hessian diagonal of Sec. 3
// (sum u(x+h) u(x-h)) and the sponge checkpoint of u^{n+1} used by the
// adjoint pass.
//
// Backward step (one launch per m = nt-1 .. 1, all shots), fused:
//   - adjoint of the discrete forward map (the back-propagated residual of
//     Sec. 2): (1 + eta dt) psi^m = 2 psi^{m+1} - (1 - eta dt) psi^{m+2}
//                                   + c2 (Lhat psi^{m+1} + dx^2 R^T a^m),
//   - reverse reconstruction of the forward field in the undamped model,
//     u^{m-2} = u^{m-1} - ((u^m - u^{m-1}) - c2 q^{m-1}), the sponge cells
//     restored from the checkpoint (leapfrog is time-reversible where eta = 0),
//   - zero-lag imaging [Sec. 2]: G += psi^m * q^{m-1}, q = Lhat u + f delta_s,
//     which is dx^2 (L u + s); the factor 2 / (v dx^2) is applied once at the
//     end (fwi_aux.cu).
//
// Work decomposition: a CTA of 128 threads owns one 64 x (8 RZ) tile of the
// padded grid and one group of shots (g, g+G, g+2G, ...); all CTAs walk their
// shots in the same order, so a shot's neighbouring tiles read each other's
// halos at about the same time and those re-reads hit L2. For each shot the
// tile (plus the stencil halo) and the point tiles the update needs are
// brought into a multi-stage shared-memory ring by TMA (cp.async.bulk.tensor)
// on mbarriers, STAGES-1 shots ahead of the compute, so HBM streams while the
// stencil runs. The tile's c2 sits in shared memory for the whole launch and
// its accumulators (illumination, offset Hessian, gradient) in registers
// across the shots; they are added to global memory (red.add) once at the
// end. Threads whose 4 x RZ points are all inside the model take a branch-free
// path (no damping, no checkpoint, no masking). Every mbarrier wait is bounded
// (~2 s of %globaltimer), after which the kernel sets ST_TIMEOUT and returns.
#include "fwi_internal.h"

#include <cudaTypedefs.h>

namespace fwi {


namespace {

// 8th-order centred second-derivative weights (the centre weight -205/72 enters
// through the -2c of each second difference)
constexpr float W1 = 8.0f / 5.0f;
constexpr float W2 = -1.0f / 5.0f;
constexpr float W3 = 8.0f / 315.0f;
constexpr float W4 = -1.0f / 560.0f;

// Lhat u at one point in second-difference form: q = sum_k W_k ((x_{-k} +
// x_{+k} - 2c) + (z_{-k} + z_{+k} - 2c)), smallest weights first. The
// differences vanish exactly for a constant field and keep the rounding of q
// relative to the field's curvature rather than to its value. The forward and
// backward kernels both call this, so q is bitwise the same in both passes.
__device__ __forceinline__ float lap8(float c, float x1, float z1, float x2, float z2, float x3,
                                     float z3, float x4, float z4)
{
    const float c2x = 2.0f * c;
    float q = W4 * ((x4 - c2x) + (z4 - c2x));
    q = fmaf(W3, (x3 - c2x) + (z3 - c2x), q);
    q = fmaf(W2, (x2 - c2x) + (z2 - c2x), q);
    q = fmaf(W1, (x1 - c2x) + (z1 - c2x), q);
    return q;
}

// One damped leapfrog step in increment form:
//   u^{n+1} = u^n + ((1 - eta dt)(u^n - u^{n-1}) + c2 q) / (1 + eta dt),
// algebraically the update of the header; carrying the small increment
// u^n - u^{n-1} keeps the FP32 rounding at the increment's scale. Written out
// in the kernels as u + fma(c2 ia, q, ((1 - e) ia)(u - u_prev)), e = eta dt,
// ia = 1/(1 + e), which is exactly u + fma(c2, q, u - u_prev) where e = 0.

// Reverse step in the model (eta = 0): u^{n-1} from u^n, u^{n+1} and q^n.
__device__ __forceinline__ float leap_back(float u, float up, float c2v, float q)
{
    return u - fmaf(-c2v, q, up - u);
}

__device__ __forceinline__ float comp(const float4 &v, int p)
{
    return p == 0 ? v.x : (p == 1 ? v.y : (p == 2 ? v.z : v.w));
}

__device__ __forceinline__ float4 lds4(const float *p) { return *reinterpret_cast<const float4 *>(p); }

// store 4 consecutive values, masking columns >= nxp
__device__ __forceinline__ void store4(float *p, int j0, int nxp, const float (&v)[4])
{
    if (j0 + 3 < nxp) {
        *reinterpret_cast<float4 *>(p) = make_float4(v[0], v[1], v[2], v[3]);
    } else {
#pragma unroll
        for (int k = 0; k < 4; ++k)
            if (j0 + k < nxp) p[k] = v[k];
    }
}

// ------------------------------------------------------------ PTX helpers
__device__ __forceinline__ uint32_t smem_u32(const void *p)
{
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}

__device__ __forceinline__ void fence_mbar_init()
{
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint32_t bar, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
}

// try_wait may suspend the thread until the phase completes or up to a
// hinted time (ns); a suspended thread issues no instructions.
__device__ __forceinline__ bool mbar_try_wait(uint32_t bar, uint32_t parity)
{
    uint32_t ok;
    asm volatile("{\n\t.reg .pred p;\n\t"
                 "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n\t"
                 "selp.u32 %0, 1, 0, p;\n\t}"
                 : "=r"(ok)
                 : "r"(bar), "r"(parity), "r"(20000u)
                 : "memory");
    return ok != 0;
}

__device__ __forceinline__ uint64_t globaltimer_ns()
{
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// Wait for phase `parity` of an mbarrier; gives up after limit_ns of
// %globaltimer (or 2^30 polls) and returns false.
__device__ __noinline__ bool mbar_wait(uint32_t bar, uint32_t parity, uint64_t limit_ns)
{
    if (mbar_try_wait(bar, parity)) return true;
    const uint64_t t0 = globaltimer_ns();
    for (uint32_t it = 0; it < (1u << 30); ++it) {
        if (mbar_try_wait(bar, parity)) return true;
        if ((it & 255u) == 255u && globaltimer_ns() - t0 > limit_ns) return false;
    }
    return false;
}

constexpr uint64_t WAIT_NS = 2000000000ull;   // per wait in normal operation
constexpr uint64_t DRAIN_NS = 200000000ull;   // per in-flight stage after a timeout

// TMA: 3-D tile (x, y, z) of a tensor map into shared memory, completion
// counted in bytes on mbarrier `bar`.
__device__ __forceinline__ void tma_load_3d(uint32_t dst, const CUtensorMap *map, int x, int y, int z,
                                            uint32_t bar)
{
    asm volatile("cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
                 " [%0], [%1, {%2, %3, %4}], [%5];" ::"r"(dst),
                 "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(z), "r"(bar)
                 : "memory");
}

constexpr int align128(int b) { return (b + 127) / 128 * 128; }

// shared-memory plan of a step kernel: mbarriers, then STAGES stages of
// NH halo tiles and NP point tiles, then EXTRA bytes
template <int TZ, int HX, int NHALO, int NPT, int STAGES, int EXTRA>
struct Ring {
    static constexpr int TXS = TX + 2 * HX;
    static constexpr int HALO = (TZ + 2 * RADIUS) * TXS; // floats of one halo tile
    static constexpr int PT = TZ * TX;                   // floats of one point tile
    static constexpr int HALO_B = align128(HALO * 4);
    static constexpr int PT_B = align128(PT * 4);
    static constexpr int STAGE_B = NHALO * HALO_B + NPT * PT_B;
    static constexpr int BAR_B = 128;
    static constexpr int SMEM = 128 + BAR_B + STAGES * STAGE_B + align128(EXTRA); // +128: base alignment
    __device__ static float *halo(unsigned char *sm, int st, int k)
    {
        return reinterpret_cast<float *>(sm + BAR_B + st * STAGE_B + k * HALO_B);
    }
    __device__ static float *point(unsigned char *sm, int st, int k)
    {
        return reinterpret_cast<float *>(sm + BAR_B + st * STAGE_B + NHALO * HALO_B + k * PT_B);
    }
    __device__ static unsigned char *extra(unsigned char *sm) { return sm + BAR_B + STAGES * STAGE_B; }
};

// Wait for the stage of pair k; false (and the CTA's abort flag set) on timeout.
template <int STAGES>
__device__ __forceinline__ bool stage_ready(uint64_t *bars, int k, int *s_abort)
{
    if (mbar_wait(smem_u32(&bars[k % STAGES]), (k / STAGES) & 1, WAIT_NS)) return true;
    *s_abort = 1;
    return false;
}

// After a timeout (seen by the whole CTA after a barrier): record it and wait,
// bounded, for the copies of pairs k+1.. still in flight, so that no TMA write
// lands in shared memory after the CTA has left.
template <int STAGES>
__device__ void abort_drain(uint64_t *bars, int k, int count, int *status)
{
    if (threadIdx.x != 0) return;
    atomicOr(status, ST_TIMEOUT);
    for (int j = k + 1; j < count && j < k + STAGES; ++j)
        mbar_wait(smem_u32(&bars[j % STAGES]), (j / STAGES) & 1, DRAIN_NS);
}

__device__ __forceinline__ unsigned char *align_smem(unsigned char *p)
{
    return reinterpret_cast<unsigned char *>((reinterpret_cast<uintptr_t>(p) + 127) & ~uintptr_t(127));
}

// order this thread's earlier generic-proxy accesses of shared memory before
// the async-proxy (TMA) writes it issues next
__device__ __forceinline__ void fence_proxy_async_smem()
{
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

} // namespace

// Per-shot scalars of one work item, fetched ahead so that their
// global-memory latency overlaps the previous item's stencil.
struct ShotScalars {
    int si, sj;    // padded cell of the source
    float amp;     // source amplitude of this time level (0 if none)
    int rb, re;    // receiver-table range of (tile, shot)
};

__device__ __forceinline__ ShotScalars fetch_scalars(const StepCommon &c, const RecTable &rt, int tile, int s,
                                                     int n_src, bool use_src, bool use_rec)
{
    ShotScalars v;
    const int2 ij = c.src_ij[s];
    v.si = ij.x;
    v.sj = ij.y;
    v.amp = use_src ? c.wav[(long long)s * c.nt + n_src] * c.src_scale : 0.f;
    v.rb = 0;
    v.re = 0;
    if (use_rec) {
        v.rb = rt.ptr[tile * c.ns + s];
        v.re = rt.ptr[tile * c.ns + s + 1];
    }
    return v;
}

// Damping of the thread's rows / columns (eta dt is separable: rows + columns)
// and where its float4 of each row sits in the per-step sponge checkpoint:
// >= 0: checkpoint index of the 4 points (contiguous, 16-byte aligned);
// -1: no sponge point; -2: mixed row (scalar path).
template <int RZ>
struct SpongeInfo {
    float ez[RZ], ex[4];
    int brow[RZ];
    __device__ void init(const Lay2D &L, int i0, int j0)
    {
#pragma unroll
        for (int r = 0; r < RZ; ++r) {
            const int d = sponge_depth(i0 + r, L.P, L.nz);
            ez[r] = L.etamax_dt * (float)(d * d) * L.inv_p2;
        }
#pragma unroll
        for (int p = 0; p < 4; ++p) {
            const int d = sponge_depth(j0 + p, L.P, L.nx);
            ex[p] = L.etamax_dt * (float)(d * d) * L.inv_p2;
        }
#pragma unroll
        for (int r = 0; r < RZ; ++r) {
            const int i = i0 + r;
            int info = -1;
            if (i < L.nzp && j0 < L.nxp) {
                bool any = false, all = true;
#pragma unroll
                for (int p = 0; p < 4; ++p) {
                    const bool inb = j0 + p < L.nxp && band_index(L, i, j0 + p) >= 0;
                    any |= inb;
                    all &= inb;
                }
                if (any) {
                    const int b0 = band_index(L, i, j0);
                    info = (all && b0 >= 0 && band_index(L, i, j0 + 3) == b0 + 3 && (b0 & 3) == 0) ? b0 : -2;
                }
            }
            brow[r] = info;
        }
    }
};

// sponge point (i, j) of the padded grid (inside the padded grid only)
__device__ __forceinline__ bool in_band(const Lay2D &L, int i, int j)
{
    return i < L.nzp && j < L.nxp && band_index(L, i, j) >= 0;
}

// index (row * 4 + column) of the thread's point that holds the source, or -1
template <int RZ>
__device__ __forceinline__ int source_slot(const ShotScalars &v, int i0, int j0)
{
    const int dr = v.si - i0, dc = v.sj - j0;
    return (dr >= 0 && dr < RZ && dc >= 0 && dc < 4) ? dr * 4 + dc : -1;
}

// load the c2 tile (TZ x TX, model + sponge cells; 0 outside) into shared memory
template <int TZ>
__device__ __forceinline__ void load_c2_tile(float *dst, const float *c2, const Lay2D &L, int bi, int bj)
{
    for (int e = threadIdx.x; e < TZ * (TX / 4); e += TPB) {
        const int r = e / (TX / 4), v = e - r * (TX / 4);
        const int i = bi + r;
        float4 val = make_float4(0.f, 0.f, 0.f, 0.f);
        if (i < L.nzp) val = __ldg(reinterpret_cast<const float4 *>(c2 + fidx(L, i, bj + 4 * v)));
        *reinterpret_cast<float4 *>(&dst[r * TX + 4 * v]) = val;
    }
}

// Lhat u of 4 consecutive points from an x-window w[-WL..WL+3] (offset WL)
// and the column values zm[k], zp[k] = rows -k, +k (k = 1..4) of each point.
#define FWI_LAP4(Q, W, WL, ZC, R)                                                                        \
    _Pragma("unroll") for (int p = 0; p < 4; ++p)                                                       \
    {                                                                                                   \
        Q[p] = lap8(W[WL + p], W[WL + p - 1] + W[WL + p + 1], comp(ZC[R + 3], p) + comp(ZC[R + 5], p),   \
                    W[WL + p - 2] + W[WL + p + 2], comp(ZC[R + 2], p) + comp(ZC[R + 6], p),             \
                    W[WL + p - 3] + W[WL + p + 3], comp(ZC[R + 1], p) + comp(ZC[R + 7], p),             \
                    W[WL + p - 4] + W[WL + p + 4], comp(ZC[R + 0], p) + comp(ZC[R + 8], p));            \
    }

// ------------------------------------------------------------ forward step
template <int RZ, int HX, bool WITH_H, int STAGES>
using FwdRing = Ring<8 * RZ, HX, 1, 1, STAGES, 8 * RZ * TX * 4>;

// grid = (tiles, groups): CTA (t, g) owns tile t and the shots g, g+G, ...;
// all CTAs walk their shots in the same order, so neighbouring tiles read
// each other's halos of the same shot at about the same time (L2 hits).
template <int RZ, int HX, bool WITH_H, int STAGES, int MINB>
__global__ void __launch_bounds__(TPB, MINB) k_fwd_step(const __grid_constant__ FwdArgs a)
{
    using R = FwdRing<RZ, HX, WITH_H, STAGES>;
    constexpr int TZ = 8 * RZ;
    constexpr int TXS = R::TXS;
    constexpr int NH = WITH_H ? HMAX_LIMIT + 1 : 1;
    constexpr int WL = WITH_H ? HMAX_LIMIT : RADIUS; // x-window left extent
    constexpr int NW = (2 * WL + 4) / 4;             // float4s in the x-window
    static_assert(!WITH_H || (RZ == 1 && HX == 12), "offset Hessian uses RZ=1, HX=12");
    extern __shared__ unsigned char smem_raw[];
    __shared__ int s_abort;
    unsigned char *smem = align_smem(smem_raw);
    uint64_t *bars = reinterpret_cast<uint64_t *>(smem);
    float *c2s = reinterpret_cast<float *>(R::extra(smem));

    const StepCommon &c = a.c;
    const Lay2D &L = c.L;
    const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
    const int tile = blockIdx.x, G = gridDim.y, g = blockIdx.y;
    const int count = (c.ns - g + G - 1) / G;
    if (count <= 0) return;
    const int bz = tile / c.ntx, bx = tile - bz * c.ntx;
    const int bi = bz * TZ, bj = bx * TX;
    const int i0 = bi + ty * RZ, j0 = bj + 4 * tx;
    // tiles with a point outside the model take the damped path in all their
    // threads (uniform per CTA); tiles inside the model the plain update
    const bool tile_sponge = bi < L.P || bi + TZ > L.P + L.nz || bj < L.P || bj + TX > L.P + L.nx;
    const bool colok = j0 < L.nxp;
    const long long nphys = (long long)L.nz * L.nx;
    const bool use_rec = a.seis != nullptr;
    SpongeInfo<RZ> sg;
    if (tile_sponge) sg.init(L, i0, j0);

    if (threadIdx.x == 0) {
        for (int k = 0; k < STAGES; ++k) mbar_init(smem_u32(&bars[k]), 1);
        fence_mbar_init();
        s_abort = 0;
    }
    load_c2_tile<TZ>(c2s, c.c2, L, bi, bj);
    __syncthreads();

    auto issue = [&](int k) {
        const int s = g + k * G;
        const int st = k % STAGES;
        const uint32_t bar = smem_u32(&bars[st]);
        fence_proxy_async_smem();
        mbar_expect_tx(bar, (R::HALO + (a.last ? 0 : R::PT)) * 4);
        tma_load_3d(smem_u32(R::halo(smem, st, 0)), &a.tm_cur, GXL + bj - HX, bi, s, bar);
        if (!a.last) tma_load_3d(smem_u32(R::point(smem, st, 0)), &a.tm_prev, GXL + bj, bi + GZ, s, bar);
    };
    if (threadIdx.x == 0)
        for (int k = 0; k < STAGES - 1 && k < count; ++k) issue(k);

    float acc_i[RZ][4];
    float acc_h[NH][4];
#pragma unroll
    for (int r = 0; r < RZ; ++r)
#pragma unroll
        for (int p = 0; p < 4; ++p) acc_i[r][p] = 0.f;
#pragma unroll
    for (int h = 0; h < NH; ++h)
#pragma unroll
        for (int p = 0; p < 4; ++p) acc_h[h][p] = 0.f;

    ShotScalars nxt = fetch_scalars(c, a.rt, tile, g, a.n, !a.last, use_rec);
    for (int k = 0; k < count; ++k) {
        if (threadIdx.x == 0 && k + STAGES - 1 < count) issue(k + STAGES - 1);
        const int s = g + k * G;
        const ShotScalars cur = nxt;
        if (k + 1 < count) nxt = fetch_scalars(c, a.rt, tile, s + G, a.n, !a.last, use_rec);
        const int st = k % STAGES;
        if (stage_ready<STAGES>(bars, k, &s_abort)) {
            const float *sm = R::halo(smem, st, 0);
            const float *pm = R::point(smem, st, 0);
            float *up = a.uprev + (long long)s * L.fstride;

            // receiver extraction d^n = R u^n
            for (int e = cur.rb + (int)threadIdx.x; e < cur.re; e += TPB) {
                const int2 en = a.rt.ent[e];
                const int zl = en.x / TX, xl = en.x - zl * TX;
                a.seis[((long long)s * c.nt + a.n) * c.nrec + en.y] = sm[(zl + RADIUS) * TXS + HX + xl];
            }
            const int sslot = source_slot<RZ>(cur, i0, j0);

            float4 zc[RZ + 2 * RADIUS];
#pragma unroll
            for (int kk = 0; kk < RZ + 2 * RADIUS; ++kk) zc[kk] = lds4(&sm[(ty * RZ + kk) * TXS + HX + 4 * tx]);

#pragma unroll
            for (int r = 0; r < RZ; ++r) {
                const float *row = &sm[(ty * RZ + r + RADIUS) * TXS + HX + 4 * tx];
                float w[4 * NW];
#pragma unroll
                for (int kk = 0; kk < NW; ++kk) {
                    const float4 t = lds4(row - WL + 4 * kk);
                    w[4 * kk] = t.x; w[4 * kk + 1] = t.y; w[4 * kk + 2] = t.z; w[4 * kk + 3] = t.w;
                }
                if (!a.last) {
                    float q[4];
                    FWI_LAP4(q, w, WL, zc, r)
#pragma unroll
                    for (int p = 0; p < 4; ++p)
                        if (sslot == r * 4 + p) q[p] += cur.amp;
                    const float4 um4 = lds4(&pm[(ty * RZ + r) * TX + 4 * tx]);
                    const float4 c24 = lds4(&c2s[(ty * RZ + r) * TX + 4 * tx]);
                    float out[4];
                    if (!tile_sponge) {
#pragma unroll
                        for (int p = 0; p < 4; ++p) {
                            const float u0 = w[WL + p];
                            out[p] = u0 + fmaf(comp(c24, p), q[p], u0 - comp(um4, p));
                        }
                        *reinterpret_cast<float4 *>(up + fidx(L, i0 + r, j0)) =
                            make_float4(out[0], out[1], out[2], out[3]);
                    } else {
                        // damped update; identical to the plain one where eta = 0
                        const int i = i0 + r;
#pragma unroll
                        for (int p = 0; p < 4; ++p) {
                            const float e = sg.ez[r] + sg.ex[p];
                            const float ia = __frcp_rn(1.0f + e);
                            const float u0 = w[WL + p];
                            out[p] = u0 + fmaf(comp(c24, p) * ia, q[p], ((1.0f - e) * ia) * (u0 - comp(um4, p)));
                        }
                        if (colok && i < L.nzp) store4(up + fidx(L, i, j0), j0, L.nxp, out);
                        if (a.band != nullptr && sg.brow[r] != -1) {
                            float *bb = a.band + ((long long)s * c.nt + a.n + 1) * L.nbandp;
                            if (sg.brow[r] >= 0) {
                                *reinterpret_cast<float4 *>(bb + sg.brow[r]) = make_float4(out[0], out[1], out[2], out[3]);
                            } else {
#pragma unroll
                                for (int p = 0; p < 4; ++p)
                                    if (in_band(L, i, j0 + p)) bb[band_index(L, i, j0 + p)] = out[p];
                            }
                        }
                    }
                    if (a.illum_utt) {
#pragma unroll
                        for (int p = 0; p < 4; ++p) {
                            const float d2 = (out[p] - 2.0f * w[WL + p]) + comp(um4, p);
                            acc_i[r][p] = fmaf(d2, d2, acc_i[r][p]);
                        }
                    }
                }
                if (!a.illum_utt) {
#pragma unroll
                    for (int p = 0; p < 4; ++p) acc_i[r][p] = fmaf(w[WL + p], w[WL + p], acc_i[r][p]);
                }
                if (WITH_H) {
#pragma unroll
                    for (int h = 0; h < NH; ++h)
                        if (h <= a.hmax) {
#pragma unroll
                            for (int p = 0; p < 4; ++p) acc_h[h][p] = fmaf(w[WL + p + h], w[WL + p - h], acc_h[h][p]);
                        }
                }
            }
        }
        __syncthreads();
        if (s_abort) {
            abort_drain<STAGES>(bars, k, count, c.status);
            return;
        }
    }

    // add this CTA's sums over its shots (model cells only)
#pragma unroll
    for (int r = 0; r < RZ; ++r) {
        const int iz = i0 + r - L.P;
#pragma unroll
        for (int p = 0; p < 4; ++p) {
            const int ix = j0 + p - L.P;
            if (iz < 0 || iz >= L.nz || ix < 0 || ix >= L.nx) continue;
            const long long o = (long long)iz * L.nx + ix;
            if (a.acc_illum != nullptr) atomicAdd(a.acc_illum + o, acc_i[r][p]);
            if (WITH_H) {
#pragma unroll
                for (int h = 0; h < NH; ++h)
                    if (h <= a.hmax) atomicAdd(a.acc_offh + h * nphys + o, acc_h[h][p]);
            }
        }
    }
}

// ----------------------------------------------------------- backward step
template <int RZ, int STAGES>
using BwdRing = Ring<8 * RZ, RADIUS, 2, 2, STAGES, 2 * 8 * RZ * TX * 4>;

template <int RZ, int STAGES, int MINB>
__global__ void __launch_bounds__(TPB, MINB) k_bwd_step(const __grid_constant__ BwdArgs a)
{
    using R = BwdRing<RZ, STAGES>;
    constexpr int TZ = 8 * RZ;
    constexpr int HX = RADIUS;
    constexpr int TXS = R::TXS;
    extern __shared__ unsigned char smem_raw[];
    __shared__ int s_abort;
    unsigned char *smem = align_smem(smem_raw);
    uint64_t *bars = reinterpret_cast<uint64_t *>(smem);
    float *c2s = reinterpret_cast<float *>(R::extra(smem));
    float *sinj = c2s + TZ * TX;

    const StepCommon &c = a.c;
    const Lay2D &L = c.L;
    const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
    const int tile = blockIdx.x, G = gridDim.y, g = blockIdx.y;
    const int count = (c.ns - g + G - 1) / G;
    if (count <= 0) return;
    const int bz = tile / c.ntx, bx = tile - bz * c.ntx;
    const int bi = bz * TZ, bj = bx * TX;
    const int i0 = bi + ty * RZ, j0 = bj + 4 * tx;
    const bool tile_sponge = bi < L.P || bi + TZ > L.P + L.nz || bj < L.P || bj + TX > L.P + L.nx;
    const bool colok = j0 < L.nxp;
    const int m = a.m;
    const bool use_rec = a.adj != nullptr;
    const bool need_band = m >= 3; // u^{m-2} in the sponge comes from checkpoint m-2 >= 1
    SpongeInfo<RZ> sg;
    if (tile_sponge) sg.init(L, i0, j0);

    if (threadIdx.x == 0) {
        for (int k = 0; k < STAGES; ++k) mbar_init(smem_u32(&bars[k]), 1);
        fence_mbar_init();
        s_abort = 0;
    }
    load_c2_tile<TZ>(c2s, c.c2, L, bi, bj);
    for (int e = threadIdx.x; e < TZ * TX; e += TPB) sinj[e] = 0.f;
    __syncthreads();

    auto issue = [&](int k) {
        const int s = g + k * G;
        const int st = k % STAGES;
        const uint32_t bar = smem_u32(&bars[st]);
        const bool need_ua = m >= 2;
        fence_proxy_async_smem();
        mbar_expect_tx(bar, (2 * R::HALO + (need_ua ? 2 : 1) * R::PT) * 4);
        tma_load_3d(smem_u32(R::halo(smem, st, 0)), &a.tm_ub, GXL + bj - HX, bi, s, bar);
        tma_load_3d(smem_u32(R::halo(smem, st, 1)), &a.tm_pa, GXL + bj - HX, bi, s, bar);
        tma_load_3d(smem_u32(R::point(smem, st, 1)), &a.tm_pb, GXL + bj, bi + GZ, s, bar);
        if (need_ua) tma_load_3d(smem_u32(R::point(smem, st, 0)), &a.tm_ua, GXL + bj, bi + GZ, s, bar);
    };
    if (threadIdx.x == 0)
        for (int k = 0; k < STAGES - 1 && k < count; ++k) issue(k);

    float acc_g[RZ][4];
#pragma unroll
    for (int r = 0; r < RZ; ++r)
#pragma unroll
        for (int p = 0; p < 4; ++p) acc_g[r][p] = 0.f;

    // adjoint-source entry of this thread for the next item (one entry per
    // thread is prefetched; further entries of a crowded tile are read late)
    auto fetch_adj = [&](const ShotScalars &v, int s, int &loc, float &val) {
        loc = -1;
        val = 0.f;
        const int e = v.rb + (int)threadIdx.x;
        if (e < v.re) {
            const int2 en = a.rt.ent[e];
            loc = en.x;
            val = a.adj[((long long)s * c.nt + m) * c.nrec + en.y] * a.adj_scale;
        }
    };

    ShotScalars cur = fetch_scalars(c, a.rt, tile, g, m - 1, true, use_rec);
    ShotScalars nxt = cur;
    if (count > 1) nxt = fetch_scalars(c, a.rt, tile, g + G, m - 1, true, use_rec);
    int adj_loc;
    float adj_val;
    fetch_adj(cur, g, adj_loc, adj_val);
    for (int k = 0; k < count; ++k) {
        if (threadIdx.x == 0 && k + STAGES - 1 < count) issue(k + STAGES - 1);
        const int s = g + k * G;
        // checkpointed sponge values of u^{m-2}, requested before the stage wait
        float4 bval[RZ];
        if (tile_sponge) {
#pragma unroll
            for (int r = 0; r < RZ; ++r) {
                bval[r] = make_float4(0.f, 0.f, 0.f, 0.f);
                if (need_band && sg.brow[r] != -1) {
                    const float *bb = a.band + ((long long)s * c.nt + (m - 2)) * L.nbandp;
                    if (sg.brow[r] >= 0) {
                        bval[r] = __ldcs(reinterpret_cast<const float4 *>(bb + sg.brow[r]));
                    } else {
                        const int i = i0 + r;
                        float t[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
                        for (int p = 0; p < 4; ++p)
                            if (in_band(L, i, j0 + p)) t[p] = __ldcs(bb + band_index(L, i, j0 + p));
                        bval[r] = make_float4(t[0], t[1], t[2], t[3]);
                    }
                }
            }
        }
        const bool has_rec = cur.rb < cur.re; // uniform over the CTA
        if (has_rec) {
            if (adj_loc >= 0) atomicAdd(&sinj[adj_loc], adj_val);
            for (int e = cur.rb + TPB + (int)threadIdx.x; e < cur.re; e += TPB) {
                const int2 en = a.rt.ent[e];
                atomicAdd(&sinj[en.x], a.adj[((long long)s * c.nt + m) * c.nrec + en.y] * a.adj_scale);
            }
        }
        // prefetch the next item's scalars (two ahead) and adjoint entry
        const ShotScalars now = cur;
        cur = nxt;
        if (k + 1 < count) {
            fetch_adj(cur, s + G, adj_loc, adj_val);
            if (k + 2 < count) nxt = fetch_scalars(c, a.rt, tile, s + 2 * G, m - 1, true, use_rec);
        }
        if (has_rec) __syncthreads();
        const int st = k % STAGES;
        if (stage_ready<STAGES>(bars, k, &s_abort)) {
            const float *su = R::halo(smem, st, 0);
            const float *sp = R::halo(smem, st, 1);
            const float *pua = R::point(smem, st, 0);
            const float *ppb = R::point(smem, st, 1);
            const long long so = (long long)s * L.fstride;
            const int sslot = source_slot<RZ>(now, i0, j0);

            float4 zu[RZ + 2 * RADIUS], zp[RZ + 2 * RADIUS];
#pragma unroll
            for (int kk = 0; kk < RZ + 2 * RADIUS; ++kk) {
                zu[kk] = lds4(&su[(ty * RZ + kk) * TXS + HX + 4 * tx]);
                zp[kk] = lds4(&sp[(ty * RZ + kk) * TXS + HX + 4 * tx]);
            }
#pragma unroll
            for (int r = 0; r < RZ; ++r) {
                const int sr = ty * RZ + r + RADIUS;
                float wu[12], wp[12];
                {
                    const float *ru = &su[sr * TXS + HX + 4 * tx];
                    const float *rp = &sp[sr * TXS + HX + 4 * tx];
                    const float4 a0 = lds4(ru - 4), a1 = lds4(ru), a2 = lds4(ru + 4);
                    const float4 b0 = lds4(rp - 4), b1 = lds4(rp), b2 = lds4(rp + 4);
                    wu[0] = a0.x; wu[1] = a0.y; wu[2] = a0.z; wu[3] = a0.w;
                    wu[4] = a1.x; wu[5] = a1.y; wu[6] = a1.z; wu[7] = a1.w;
                    wu[8] = a2.x; wu[9] = a2.y; wu[10] = a2.z; wu[11] = a2.w;
                    wp[0] = b0.x; wp[1] = b0.y; wp[2] = b0.z; wp[3] = b0.w;
                    wp[4] = b1.x; wp[5] = b1.y; wp[6] = b1.z; wp[7] = b1.w;
                    wp[8] = b2.x; wp[9] = b2.y; wp[10] = b2.z; wp[11] = b2.w;
                }
                // q^{m-1} = Lhat u^{m-1} + f(t_{m-1}) delta_s (as in the forward step m-1)
                float qu[4], qp[4];
                FWI_LAP4(qu, wu, 4, zu, r)
                FWI_LAP4(qp, wp, 4, zp, r)
#pragma unroll
                for (int p = 0; p < 4; ++p)
                    if (sslot == r * 4 + p) qu[p] += now.amp;
                if (has_rec) {
                    const float4 inj = lds4(&sinj[(ty * RZ + r) * TX + 4 * tx]);
#pragma unroll
                    for (int p = 0; p < 4; ++p) qp[p] += comp(inj, p);
                }
                const float4 ua4 = lds4(&pua[(ty * RZ + r) * TX + 4 * tx]);
                const float4 pb4 = lds4(&ppb[(ty * RZ + r) * TX + 4 * tx]);
                const float4 c24 = lds4(&c2s[(ty * RZ + r) * TX + 4 * tx]);
                float unew[4], pnew[4];
                if (!tile_sponge) {
#pragma unroll
                    for (int p = 0; p < 4; ++p) {
                        const float p1 = wp[4 + p], u1 = wu[4 + p], c2v = comp(c24, p);
                        pnew[p] = p1 + fmaf(c2v, qp[p], p1 - comp(pb4, p));
                        acc_g[r][p] = fmaf(pnew[p], qu[p], acc_g[r][p]);
                        unew[p] = leap_back(u1, comp(ua4, p), c2v, qu[p]);
                    }
                    *reinterpret_cast<float4 *>(a.pb + so + fidx(L, i0 + r, j0)) =
                        make_float4(pnew[0], pnew[1], pnew[2], pnew[3]);
                    if (m >= 2)
                        *reinterpret_cast<float4 *>(a.ua + so + fidx(L, i0 + r, j0)) =
                            make_float4(unew[0], unew[1], unew[2], unew[3]);
                } else {
                    const int i = i0 + r;
#pragma unroll
                    for (int p = 0; p < 4; ++p) {
                        const int j = j0 + p;
                        const float e = sg.ez[r] + sg.ex[p];
                        const float ia = __frcp_rn(1.0f + e);
                        const float p1 = wp[4 + p], u1 = wu[4 + p], c2v = comp(c24, p);
                        const bool valid = i < L.nzp && j < L.nxp;
                        pnew[p] = p1 + fmaf(c2v * ia, qp[p], ((1.0f - e) * ia) * (p1 - comp(pb4, p)));
                        if (valid) acc_g[r][p] = fmaf(pnew[p], qu[p], acc_g[r][p]);
                        unew[p] = (valid && band_index(L, i, j) >= 0) ? comp(bval[r], p)
                                                                       : leap_back(u1, comp(ua4, p), c2v, qu[p]);
                    }
                    if (colok && i < L.nzp) {
                        store4(a.pb + so + fidx(L, i, j0), j0, L.nxp, pnew);
                        if (m >= 2) store4(a.ua + so + fidx(L, i, j0), j0, L.nxp, unew);
                    }
                }
            }
        }
        __syncthreads();
        if (s_abort) {
            abort_drain<STAGES>(bars, k, count, c.status);
            return;
        }
        if (has_rec) {
            for (int e = now.rb + (int)threadIdx.x; e < now.re; e += TPB) sinj[a.rt.ent[e].x] = 0.f;
            __syncthreads();
        }
    }

    // add this CTA's sum over its shots (padded grid)
#pragma unroll
    for (int r = 0; r < RZ; ++r) {
        const int i = i0 + r;
#pragma unroll
        for (int p = 0; p < 4; ++p) {
            const int j = j0 + p;
            if (i < L.nzp && j < L.nxp) atomicAdd(a.acc_grad + (long long)i * L.nxp + j, acc_g[r][p]);
        }
    }
}

// ---------------------------------------------------------------- launchers
namespace {
#ifndef FWI_F_ST
#define FWI_F_ST 3
#endif
#ifndef FWI_H_ST
#define FWI_H_ST 4
#endif
#ifndef FWI_B_ST
#define FWI_B_ST 3
#endif
#ifndef FWI_F_MINB
#define FWI_F_MINB 3
#endif
#ifndef FWI_B_MINB
#define FWI_B_MINB 3
#endif
// forward without the offset Hessian: 64 x 32 tiles
constexpr int F_RZ = 4, F_ST = FWI_F_ST, F_MINB = FWI_F_MINB;
// forward with the offset Hessian: 64 x 8 tiles, halo 12
constexpr int H_RZ = 1, H_ST = FWI_H_ST, H_MINB = 3;
// backward: 64 x 16 tiles
constexpr int B_RZ = 2, B_ST = FWI_B_ST, B_MINB = FWI_B_MINB;

#define K_FWD k_fwd_step<F_RZ, RADIUS, false, F_ST, F_MINB>
#define K_FWDH k_fwd_step<H_RZ, HMAX_LIMIT, true, H_ST, H_MINB>
#define K_BWD k_bwd_step<B_RZ, B_ST, B_MINB>
constexpr int SMEM_FWD = FwdRing<F_RZ, RADIUS, false, F_ST>::SMEM;
constexpr int SMEM_FWDH = FwdRing<H_RZ, HMAX_LIMIT, true, H_ST>::SMEM;
constexpr int SMEM_BWD = BwdRing<B_RZ, B_ST>::SMEM;

int g_occ[3] = {0, 0, 0};

void prepare_kernels()
{
    static bool done = false;
    if (done) return;
    done = true;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) {
        cudaGetLastError();
        g_occ[0] = g_occ[1] = g_occ[2] = 2;
        return;
    }
    cudaFuncSetAttribute(K_FWD, cudaFuncAttributeMaxDynamicSharedMemorySize, SMEM_FWD);
    cudaFuncSetAttribute(K_FWDH, cudaFuncAttributeMaxDynamicSharedMemorySize, SMEM_FWDH);
    cudaFuncSetAttribute(K_BWD, cudaFuncAttributeMaxDynamicSharedMemorySize, SMEM_BWD);
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&g_occ[0], K_FWD, TPB, SMEM_FWD) != cudaSuccess) g_occ[0] = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&g_occ[1], K_FWDH, TPB, SMEM_FWDH) != cudaSuccess) g_occ[1] = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&g_occ[2], K_BWD, TPB, SMEM_BWD) != cudaSuccess) g_occ[2] = 0;
    cudaGetLastError();
    for (int k = 0; k < 3; ++k)
        if (g_occ[k] < 1) g_occ[k] = 2;
}

int sm_count_dev()
{
    static int n = -1;
    if (n < 0) {
        int dev = 0, v = 0;
        if (cudaGetDevice(&dev) == cudaSuccess &&
            cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev) == cudaSuccess && v > 0)
            n = v;
        else {
            cudaGetLastError();
            n = 152;
        }
    }
    return n;
}
} // namespace

void step_boxes(StepKind kind, int &hx, int &hy, int &px, int &py)
{
    int rz = kind == STEP_FWD ? F_RZ : (kind == STEP_FWD_OFFH ? H_RZ : B_RZ);
    int halo = kind == STEP_FWD_OFFH ? HMAX_LIMIT : RADIUS;
    hx = TX + 2 * halo;
    hy = 8 * rz + 2 * RADIUS;
    px = TX;
    py = 8 * rz;
}

Tiling make_tiling(const Lay2D &L, int ns, StepKind kind)
{
    prepare_kernels();
    Tiling t;
    int hx, hy, px, py;
    step_boxes(kind, hx, hy, px, py);
    t.tz = py;
    t.ntx = (L.nxp + TX - 1) / TX;
    t.ntz = (L.nzp + t.tz - 1) / t.tz;
    const int tiles = t.ntx * t.ntz;
    const int slots = sm_count_dev() * g_occ[kind];
    int groups = slots / tiles;
    if (groups < 1) groups = 1;
    if (groups > ns) groups = ns;
    t.groups = groups;
    return t;
}

cudaError_t launch_fwd_step(const FwdArgs &a, const Tiling &t, bool with_offh, cudaStream_t st)
{
    if (with_offh)
        K_FWDH<<<dim3(t.ntx * t.ntz, t.groups), TPB, SMEM_FWDH, st>>>(a);
    else
        K_FWD<<<dim3(t.ntx * t.ntz, t.groups), TPB, SMEM_FWD, st>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_bwd_step(const BwdArgs &a, const Tiling &t, cudaStream_t st)
{
    K_BWD<<<dim3(t.ntx * t.ntz, t.groups), TPB, SMEM_BWD, st>>>(a);
    return cudaGetLastError();
}

// Tensor map over `nfields` stored fields [nfields][rows][pitch] (float32)
// with a box of bx x by cells; out-of-range cells read as zero.
bool encode_field_map(CUtensorMap *map, const float *base, const Lay2D &L, int nfields, int bx, int by)
{
    static PFN_cuTensorMapEncodeTiled_v12000 encode = nullptr;
    if (!encode) {
        cudaDriverEntryPointQueryResult q;
        void *fn = nullptr;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q) !=
                cudaSuccess ||
            q != cudaDriverEntryPointSuccess || !fn)
            return false;
        encode = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(fn);
    }
    const cuuint64_t dims[3] = {(cuuint64_t)L.pitch, (cuuint64_t)L.rows, (cuuint64_t)nfields};
    const cuuint64_t strides[2] = {(cuuint64_t)L.pitch * sizeof(float), (cuuint64_t)L.fstride * sizeof(float)};
    const cuuint32_t box[3] = {(cuuint32_t)bx, (cuuint32_t)by, 1};
    const cuuint32_t estr[3] = {1, 1, 1};
    CUresult r = encode(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, const_cast<float *>(base), dims, strides, box,
                        estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                        CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS;
}

} // namespace fwi
