// fwi_step2d.cu -- time-step kernels of the 2-D FWI gradient (sm_103a).
//
// Forward step (one launch per time level n, all shots):
//   (1 + eta dt) u^{n+1} = 2 u^n - (1 - eta dt) u^{n-1} + c2 (Lhat u^n + f_s(t_n) delta_s)
// with c2 = (v dt/dx)^2 and Lhat the 8th-order Laplacian without 1/dx^2: the
// leapfrog discretisation of the constant-density acoustic equation of Sec. 2
// with an absorbing sponge u_tt + 2 eta u_t. Fused into the same pass over the
// tile: receiver extraction d^n = R u^n [Sec. 2], the shot illumination of
// Eq. 1 (sum u^2, or the u_tt^2 form), the sponge checkpoint of u^{n+1} used
// by the adjoint pass and, in the fused offset-Hessian variants, the
// offset-Hessian diagonal of Sec. 3 (sum u(x+h) u(x-h)); the split variants
// leave that sum to k_offh_level, launched after the plain step of each level
// (the autotuner keeps whichever is faster for the problem).
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
// Work decomposition: the (tile, shot) pairs of one time level, cut into
// chunks of a few shots of one 64 x (8 RZ) tile, are handed out in order by
// an atomic counter to one CTA (128 threads) per resident slot: the load is
// balanced whatever a tile costs (sponge and receiver tiles do more), and at
// any moment all CTAs work on neighbouring tiles of the same shots, whose
// halo re-reads then hit L2. Thread 0 stages item descriptors a few items
// ahead; for each item the tile (plus the stencil halo) and the point tiles
// the update needs are brought into a multi-stage shared-memory ring by TMA
// (cp.async.bulk.tensor) on mbarriers, STAGES-1 items ahead of the compute,
// so HBM streams while the stencil runs. The tile's c2 sits in shared memory
// and its accumulators (illumination, offset Hessian, gradient) in registers
// for the chunk; they are added to global memory (red.add) at each tile
// change. Threads whose 4 x RZ points are all inside the model take a branch-free
// path (no damping, no checkpoint, no masking). Every mbarrier wait is bounded
// (~2 s of %globaltimer), after which the kernel sets ST_TIMEOUT and returns.
#include "fwi_device.cuh"

#include <cudaTypedefs.h>

#include <algorithm>
#include <map>
#include <mutex>
#include <tuple>

namespace fwi {



// ------------------------------------------------------------- scheduling
// The work of one launch is the (tile, shot) pairs. They are cut into chunks
// of S shots of one tile; chunk q covers tile q % ntiles and shots
// [(q / ntiles) S, (q / ntiles) S + S). One CTA per resident slot takes chunks
// in order from an atomic counter, so the load is balanced whatever a tile
// costs, and at any moment all CTAs work on nearby chunks: neighbouring tiles
// of the same shots, whose halo re-reads then hit L2.
struct alignas(16) ItemDesc {
    int tile, s;   // tile and (first) shot of the item; tile < 0: no more work
    int rb, re;    // receiver-table range of (tile, shot)
    int si, sj;    // padded cell of the shot's source (8-byte aligned pair)
    float amp;     // source amplitude at this time level
    int model;     // model of the item in a batched launch
    int nsh;       // shots in the item (items of two shots: shots s, s + 1)
    float amp1;    // the second shot's amplitude, source cell and receivers
    int si1, sj1;
    int rb1, re1;
    int pad[2];
};

// State of the staging lane that walks the CTA's chunks.
struct Cursor {
    int model, tile, s, s_end; // current chunk
    int q_next;                // next chunk, taken one chunk ahead (-1: none)
    bool done;
};

__device__ __forceinline__ int grab_chunk(int *counter, int nchunks)
{
    const int q = atomicAdd(counter, 1);
    return q < nchunks ? q : -1;
}

// chunk q of a launch: its model (chunks of the models are consecutive),
// tile and shot range
template <class BT>
__device__ __forceinline__ void cursor_set(Cursor &cu, int q, const BT &B)
{
    int m = 0;
#pragma unroll
    for (int k = 0; k + 1 < BT::NM; ++k)
        if (k + 1 < B.nm && q >= B.chunk_end[k]) m = k + 1;
    const StepCommon &c = B.m[m].c;
    const int ntiles = c.ntx * c.ntz;
    const int local = q - (m > 0 ? B.chunk_end[m - 1] : 0);
    const int blk = local / ntiles;
    cu.model = m;
    cu.tile = local - blk * ntiles;
    // shot blocks of `chunk` shots; of two or more, the last block of the
    // model is cut in two (the level's last chunks are shorter, so the CTAs
    // run out of work closer together)
    const int nb = (c.ns + B.chunk - 1) / B.chunk;
    if (blk < nb - 1 || nb == 1) {
        cu.s = blk * B.chunk;
        cu.s_end = min(c.ns, cu.s + B.chunk);
    } else {
        const int s0 = (nb - 1) * B.chunk, h = (c.ns - s0 + 1) / 2;
        cu.s = blk == nb - 1 ? s0 : s0 + h;
        cu.s_end = blk == nb - 1 ? s0 + h : c.ns;
    }
}

template <class BT>
__device__ __forceinline__ void cursor_init(Cursor &cu, const BT &B)
{
    const int nchunks = B.chunk_end[B.nm - 1];
    const int q = grab_chunk(B.sched, nchunks);
    cu.done = q < 0;
    cu.q_next = -1;
    cu.model = cu.tile = cu.s = cu.s_end = 0;
    if (!cu.done) {
        cursor_set(cu, q, B);
        cu.q_next = grab_chunk(B.sched, nchunks);
    }
}

// next (model, tile, shots s .. s + cnt - 1 with cnt <= spi) of this CTA;
// false when the launch's work is exhausted
template <class BT>
__device__ __forceinline__ bool cursor_next(Cursor &cu, const BT &B, int &model, int &tile, int &s, int spi, int &cnt)
{
    if (cu.done) return false;
    if (cu.s >= cu.s_end) {
        if (cu.q_next < 0) {
            cu.done = true;
            return false;
        }
        cursor_set(cu, cu.q_next, B);
        cu.q_next = grab_chunk(B.sched, B.chunk_end[B.nm - 1]);
    }
    model = cu.model;
    tile = cu.tile;
    s = cu.s;
    cnt = min(spi, cu.s_end - cu.s);
    cu.s += cnt;
    return true;
}

__device__ __forceinline__ void cp_async4(void *dst, const void *src)
{
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(smem_u32(dst)), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async8(void *dst, const void *src)
{
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(smem_u32(dst)), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;" ::: "memory"); }

__device__ __forceinline__ bool has_rec(const FwdArgs &a) { return a.seis != nullptr; }
__device__ __forceinline__ bool has_rec(const BwdArgs &a) { return a.adj != nullptr; }
__device__ __forceinline__ bool has_rec(const BornArgs &a) { return a.dseis != nullptr; }

// Stage the descriptor of the CTA's next item into a ring slot (lane 0 of
// warp 1 only): model, tile and shot from the chunk cursor (shared memory),
// the per-shot scalars (source cell, amplitude, receiver range) copied from
// global memory by cp.async, so that no register holds them while the loads
// are in flight. The copies complete at cp_async_wait_all(), which the
// staging thread calls before the barrier that publishes the slot. The
// amplitude is stored unscaled (times src_scale at use).
template <int SPI, class BT>
__device__ __forceinline__ void stage_desc_async(ItemDesc *slot, Cursor &cu, const BT &B, int n_src, bool use_src)
{
    int mdl = 0, t = -1, s = 0, cnt = 0;
    if (!cursor_next(cu, B, mdl, t, s, SPI, cnt)) t = -1;
    slot->tile = t;
    slot->s = s;
    slot->model = mdl;
    slot->nsh = cnt;
    if (t < 0) {
        slot->rb = slot->re = slot->si = slot->sj = 0;
        slot->amp = 0.f;
        return;
    }
    const auto &a = B.m[mdl];
    const StepCommon &c = a.c;
    cp_async8(&slot->si, &c.src_ij[s]);
    if (use_src)
        cp_async4(&slot->amp, &c.wav[(long long)s * c.nt + n_src]);
    else
        slot->amp = 0.f;
    if (has_rec(a)) {
        cp_async4(&slot->rb, &a.rt.ptr[t * c.ns + s]);
        cp_async4(&slot->re, &a.rt.ptr[t * c.ns + s + 1]);
    } else {
        slot->rb = slot->re = 0;
    }
    if (SPI > 1) {
        if (cnt > 1) {
            cp_async8(&slot->si1, &c.src_ij[s + 1]);
            if (use_src)
                cp_async4(&slot->amp1, &c.wav[(long long)(s + 1) * c.nt + n_src]);
            else
                slot->amp1 = 0.f;
            if (has_rec(a)) {
                cp_async4(&slot->rb1, &a.rt.ptr[t * c.ns + s + 1]);
                cp_async4(&slot->re1, &a.rt.ptr[t * c.ns + s + 2]);
            } else {
                slot->rb1 = slot->re1 = 0;
            }
        } else {
            slot->si1 = slot->sj1 = -1000000;
            slot->amp1 = 0.f;
            slot->rb1 = slot->re1 = 0;
        }
    }
}

// After a timeout (seen by the whole CTA after a barrier): record it and wait,
// bounded, for the copies of item k and of the items after it that were
// issued, so that no TMA write lands in shared memory after the CTA has left.
template <int STAGES>
__device__ void abort_drain_ring(uint64_t *bars, const ItemDesc *desc, int k, int *status)
{
    if (threadIdx.x != 0) return;
    atomicOr(status, ST_TIMEOUT);
    for (int j = k; j < k + STAGES; ++j)
        if (desc[j % DESC_RING].tile >= 0) mbar_wait(smem_u32(&bars[j % STAGES]), (j / STAGES) & 1, DRAIN_NS);
}

// Where the thread's float4 of each row sits in the per-step sponge
// checkpoint: >= 0: checkpoint index of the 4 points (contiguous, 16-byte
// aligned); -1: no sponge point; -2: mixed row (scalar path).
template <int RZ>
struct SpongeInfo {
    int brow[RZ];
    __device__ void init(const Lay2D &L, int i0, int j0)
    {
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
__device__ __forceinline__ int source_slot(int si, int sj, int i0, int j0)
{
    const int dr = si - i0, dc = sj - j0;
    return (dr >= 0 && dr < RZ && dc >= 0 && dc < 4) ? dr * 4 + dc : -1;
}
template <int RZ>
__device__ __forceinline__ int source_slot(const ItemDesc &v, int i0, int j0)
{
    return source_slot<RZ>(v.si, v.sj, i0, j0);
}

// N TZ x TX tiles of field-layout coefficient arrays (c2, damping, the planes
// of D~) into shared memory (0 below the padded grid; a null source is
// skipped). Every load is issued before the first store, so that a tile
// change waits for one memory latency rather than one per tile.
template <int TZ, int N>
__device__ __forceinline__ void load_tiles(float *(&dst)[N], const float *(&src)[N], const Lay2D &L, int bi, int bj)
{
    constexpr int PER = TZ * (TX / 4), NV = (PER + TPB - 1) / TPB; // float4s of one tile, per thread
    float4 v[N][NV];
#pragma unroll
    for (int e = 0; e < N; ++e)
#pragma unroll
        for (int q = 0; q < NV; ++q) {
            const int idx = threadIdx.x + q * TPB, r = idx / (TX / 4), c4 = idx - r * (TX / 4);
            v[e][q] = make_float4(0.f, 0.f, 0.f, 0.f);
            if (src[e] != nullptr && (PER % TPB == 0 || idx < PER) && bi + r < L.nzp)
                v[e][q] = __ldg(reinterpret_cast<const float4 *>(src[e] + fidx(L, bi + r, bj + 4 * c4)));
        }
#pragma unroll
    for (int e = 0; e < N; ++e)
#pragma unroll
        for (int q = 0; q < NV; ++q) {
            const int idx = threadIdx.x + q * TPB, r = idx / (TX / 4), c4 = idx - r * (TX / 4);
            if (src[e] != nullptr && (PER % TPB == 0 || idx < PER))
                *reinterpret_cast<float4 *>(&dst[e][r * TX + 4 * c4]) = v[e][q];
        }
}

// c2 and (in sponge tiles) the damping factor of one tile
template <int TZ>
__device__ __forceinline__ void load_coef_tiles(float *c2s, float *dms, const StepCommon &c, bool sponge, int bi,
                                                int bj)
{
    float *dst[2] = {c2s, dms};
    const float *src[2] = {c.c2, sponge ? c.damp : nullptr};
    load_tiles<TZ, 2>(dst, src, c.L, bi, bj);
}

// ------------------------------------------------------------ forward step
// a stage holds SPI consecutive shots' halo tiles and point tiles (one TMA
// box of depth SPI in the shot dimension each; the tile sizes are multiples
// of 128 bytes, so the shots' tiles are contiguous)
template <int RZ, int HX, bool WITH_H, int STAGES, int SPI = 1>
using FwdRing = Ring<8 * RZ, HX, SPI, SPI, STAGES, 2 * 8 * RZ * TX * 4>; // + c2 and damping tiles

// NHC: offsets h = 0 .. NHC-1 of the offset Hessian are accumulated (any
// hmax <= NHC-1; offsets above hmax are computed and not stored)
// QOUT (segments re-propagated from snapshots): also store q^n = Lhat u^n +
// f delta_s at a.qout, and u^{n+1} only where a.uout is not null
template <int RZ, int HX, bool WITH_H, int STAGES, int MINB, int NM, int SPI = 1, int NHC = HMAX_LIMIT + 1,
          bool QOUT = false>
__global__ void __launch_bounds__(TPB, MINB) k_fwd_step(const __grid_constant__ Batch<FwdArgs, NM> B)
{
    static_assert(!QOUT || (!WITH_H && NM == 1), "q output: plain forward step of one model");
    using R = FwdRing<RZ, HX, WITH_H, STAGES, SPI>;
    static_assert(SPI == 1 || R::HALO_B == R::HALO * 4, "contiguous shot tiles");
    constexpr int TZ = 8 * RZ;
    constexpr int TXS = R::TXS;
    constexpr int NH = WITH_H ? NHC : 1;
    static_assert(NHC >= 1 && NHC <= HMAX_LIMIT + 1, "offset count");
    constexpr int WL = WITH_H ? HMAX_LIMIT : RADIUS; // x-window left extent
    constexpr int NW = (2 * WL + 4) / 4;             // float4s in the x-window
    constexpr int D = STAGES - 1;                    // items in flight ahead of the compute
    static_assert(!WITH_H || (RZ == 1 && HX == 12), "offset Hessian uses RZ=1, HX=12");
    // item j's descriptor is staged (lane 0 of warp 1) in iteration j-D-1
    // and read in iteration j-D (copy issue) and j-1 (prefetch) and j: always
    // at least one barrier after it was written, for any D >= 1
    static_assert(D >= 1 && D + 2 <= DESC_RING, "needs 2 <= STAGES <= 7");
    // live descriptor slots in iteration k: k .. k+D+1 (read, issued, staged)
    extern __shared__ unsigned char smem_raw[];
    __shared__ int s_abort;
    __shared__ ItemDesc s_desc[DESC_RING];
    unsigned char *smem = align_smem(smem_raw);
    uint64_t *bars = reinterpret_cast<uint64_t *>(smem);
    float *c2s = reinterpret_cast<float *>(R::extra(smem));
    float *dms = c2s + 8 * RZ * TX; // damping tile (sponge tiles)

    // launch-wide values (time level, flags) are those of model 0
    const FwdArgs &a0 = B.m[0];
    const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;

    if (threadIdx.x == 0) {
        for (int k = 0; k < STAGES; ++k) mbar_init(smem_u32(&bars[k]), 1);
        fence_mbar_init();
        s_abort = 0;
    }
    __syncthreads();

    // lane 0 of warp 1 walks the chunks (cursor in shared memory) and stages
    // descriptors D + 1 items ahead
    __shared__ Cursor s_cu;
    auto stage = [&](int slot) { stage_desc_async<SPI>(&s_desc[slot % DESC_RING], s_cu, B, a0.n, !a0.last); };
    auto issue = [&](const ItemDesc &d, int k) {
        const FwdArgs &ad = B.m[NM == 1 ? 0 : d.model];
        const int bz = d.tile / ad.c.ntx, bx = d.tile - bz * ad.c.ntx;
        const int st = k % STAGES;
        const uint32_t bar = smem_u32(&bars[st]);
        fence_proxy_async_smem();
        mbar_expect_tx(bar, SPI * (R::HALO + (a0.last ? 0 : R::PT)) * 4);
        tma_load_3d(smem_u32(R::halo(smem, st, 0)), &ad.tm_cur, GXL + bx * TX - HX, bz * TZ, d.s, bar);
        if (!a0.last)
            tma_load_3d(smem_u32(R::point(smem, st, 0)), &ad.tm_prev, GXL + bx * TX, bz * TZ + GZ, d.s, bar);
    };
    // lane 0 of warp 1 walks the chunks and stages descriptors; thread 0
    // issues the copies of a descriptor staged one barrier earlier
    if (threadIdx.x == 32) {
        cursor_init(s_cu, B);
        for (int k = 0; k <= D; ++k) stage(k);
        cp_async_wait_all();
    }
    __syncthreads();
    if (threadIdx.x == 0)
        for (int k = 0; k < D; ++k)
            if (s_desc[k].tile >= 0) issue(s_desc[k], k);

    float2 acc_i[RZ][2];
    // offset Hessian of the thread's points 0..3: even h: [0] = (0, 1), [1] = (2, 3);
    // odd h: [0] = (1, 2), [1] = (0, 3)
    float2 acc_h[NH][2];
    int cur_tile = -1, cur_model = 0, bi = 0, bj = 0, i0 = 0, j0 = 0;
    bool tile_sponge = false, colok = false;
    SpongeInfo<RZ> sg;

    // accumulators of the current tile to global memory
    auto flush = [&]() {
        const FwdArgs &a = B.m[NM == 1 ? 0 : cur_model];
        const Lay2D &L = a.c.L;
        const long long nphys = (long long)L.nz * L.nx;
#pragma unroll
        for (int r = 0; r < RZ; ++r) {
            const int iz = i0 + r - L.P, ix0 = j0 - L.P;
            if (((L.P | L.nx) & 3) == 0 && iz >= 0 && iz < L.nz && ix0 >= 0 && ix0 + 3 < L.nx) {
                // the thread's 4 points inside the model, 16-byte aligned: one
                // vector reduction per sum
                const long long o = (long long)iz * L.nx + ix0;
                if (a.acc_illum != nullptr)
                    red_add4(a.acc_illum + o, acc_i[r][0].x, acc_i[r][0].y, acc_i[r][1].x, acc_i[r][1].y);
                if (WITH_H) {
#pragma unroll
                    for (int h = 0; h < NH; ++h)
                        if (h <= a0.hmax) {
                            if (h & 1)
                                red_add4(a.acc_offh + h * nphys + o, acc_h[h][1].x, acc_h[h][0].x, acc_h[h][0].y,
                                         acc_h[h][1].y);
                            else
                                red_add4(a.acc_offh + h * nphys + o, acc_h[h][0].x, acc_h[h][0].y, acc_h[h][1].x,
                                         acc_h[h][1].y);
                        }
                }
                continue;
            }
#pragma unroll
            for (int p = 0; p < 4; ++p) {
                const int ix = j0 + p - L.P;
                if (iz < 0 || iz >= L.nz || ix < 0 || ix >= L.nx) continue;
                const long long o = (long long)iz * L.nx + ix;
                if (a.acc_illum != nullptr)
                    atomicAdd(a.acc_illum + o, p < 2 ? (p == 0 ? acc_i[r][0].x : acc_i[r][0].y)
                                                     : (p == 2 ? acc_i[r][1].x : acc_i[r][1].y));
                if (WITH_H) {
#pragma unroll
                    for (int h = 0; h < NH; ++h)
                        if (h <= a0.hmax)
                            atomicAdd(a.acc_offh + h * nphys + o,
                                      (h & 1) ? (p == 0 ? acc_h[h][1].x : p == 1 ? acc_h[h][0].x
                                                 : p == 2 ? acc_h[h][0].y : acc_h[h][1].y)
                                              : ((p & 1) ? acc_h[h][p >> 1].y : acc_h[h][p >> 1].x));
                }
            }
        }
    };

    int k = 0;
    for (;; ++k) {
        if (threadIdx.x == 0) {
            const ItemDesc d = s_desc[(k + D) % DESC_RING];
            if (d.tile >= 0) issue(d, k + D);
        } else if (threadIdx.x == 32) {
            stage(k + D + 1);
        }
        const ItemDesc now = s_desc[k % DESC_RING];
        if (now.tile < 0) {
            if (threadIdx.x == 32) cp_async_wait_all(); // (none in flight once the cursor is done)
            break;
        }
        const int s = now.s;
        const int mi = NM == 1 ? 0 : now.model;
        const FwdArgs &a = B.m[mi];
        const StepCommon &c = a.c;
        const Lay2D &L = c.L;
        if (now.tile != cur_tile || mi != cur_model) {
            if (cur_tile >= 0) flush();
            cur_tile = now.tile;
            cur_model = mi;
            const int bz = cur_tile / c.ntx, bx = cur_tile - bz * c.ntx;
            bi = bz * TZ;
            bj = bx * TX;
            i0 = bi + ty * RZ;
            j0 = bj + 4 * tx;
            // tiles with a point outside the model take the damped path in
            // all their threads (uniform per CTA); inside the model the plain update
            tile_sponge = bi < L.P || bi + TZ > L.P + L.nz || bj < L.P || bj + TX > L.P + L.nx;
            colok = j0 < L.nxp;
            if (tile_sponge) sg.init(L, i0, j0);
#pragma unroll
            for (int r = 0; r < RZ; ++r) acc_i[r][0] = acc_i[r][1] = make_float2(0.f, 0.f);
#pragma unroll
            for (int h = 0; h < NH; ++h) acc_h[h][0] = acc_h[h][1] = make_float2(0.f, 0.f);
            load_coef_tiles<TZ>(c2s, dms, c, tile_sponge, bi, bj);
            __syncthreads();
        }
        const int st = k % STAGES;
        const bool ready = stage_ready<STAGES>(bars, k, &s_abort);
        // receiver extraction d^n = R u^n of the item's shots: the entries of
        // (tile, s) and (tile, s + 1) are consecutive in the receiver table.
        // One warp-uniform test skips the (common) tiles without receivers.
        const int rend = (SPI > 1 && now.nsh > 1) ? now.re1 : now.re;
        if (ready && rend > now.rb) {
#pragma unroll 1
            for (int e = now.rb + (int)threadIdx.x; e < rend; e += TPB) {
                const int2 en = a.rt.ent[e];
                const int sh = (SPI > 1 && e >= now.re) ? 1 : 0;
                const int zl = en.x / TX, xl = en.x - zl * TX;
                a.seis[((long long)(s + sh) * c.nt + a.n) * c.nrec + en.y] =
                    R::halo(smem, st, sh)[(zl + RADIUS) * TXS + HX + xl];
            }
        }
        // the item's shots, one after the other (accumulators are shared)
#pragma unroll 1
        for (int sh = 0; sh < SPI && ready; ++sh) {
            if (sh >= now.nsh) break; // uniform
            const int ss = s + sh;
            const float *sm = R::halo(smem, st, sh);
            const float *pm = R::point(smem, st, sh);
            float *up = a.uout + (long long)ss * L.fstride;

            // the shot's source cell, if it lies in this tile (warp-uniform)
            const int si = sh == 0 ? now.si : now.si1, sj = sh == 0 ? now.sj : now.sj1;
            const bool src_tile = (unsigned)(si - bi) < (unsigned)TZ && (unsigned)(sj - bj) < (unsigned)TX;
            const int sslot = src_tile ? source_slot<RZ>(si, sj, i0, j0) : -1;

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
                const float2 u0[2] = {f2(w[WL], w[WL + 1]), f2(w[WL + 2], w[WL + 3])};
                if (!a.last) {
                    float2 q[2];
                    lap4<WL>(q, w, zc, r);
                    if (src_tile) {
                        const float amp = (sh == 0 ? now.amp : now.amp1) * c.src_scale;
                        if (sslot == r * 4 + 0) q[0].x += amp;
                        if (sslot == r * 4 + 1) q[0].y += amp;
                        if (sslot == r * 4 + 2) q[1].x += amp;
                        if (sslot == r * 4 + 3) q[1].y += amp;
                    }
                    const float4 um4 = lds4(&pm[(ty * RZ + r) * TX + 4 * tx]);
                    const float4 c24 = lds4(&c2s[(ty * RZ + r) * TX + 4 * tx]);
                    float2 out[2];
                    if constexpr (QOUT) {
                        // in place of u^{n-1}: this thread read its points' u^{n-1} (um4) above
                        const int i = i0 + r;
                        const float qv[4] = {q[0].x, q[0].y, q[1].x, q[1].y};
                        if (colok && i < L.nzp)
                            store4(a.qout + (long long)ss * L.fstride + fidx(L, i, j0), j0, L.nxp, qv);
                    }
                    if (!tile_sponge) {
#pragma unroll
                        for (int h = 0; h < 2; ++h)
                            out[h] = add2(u0[h], fma2(half2of(c24, h), q[h], sub2(u0[h], half2of(um4, h))));
                        if (!QOUT || a.uout != nullptr)
                            *reinterpret_cast<float4 *>(up + fidx(L, i0 + r, j0)) =
                                make_float4(out[0].x, out[0].y, out[1].x, out[1].y);
                    } else {
                        // damped update; identical to the plain one where eta = 0
                        const int i = i0 + r;
                        const float4 ia4 = lds4(&dms[(ty * RZ + r) * TX + 4 * tx]);
#pragma unroll
                        for (int h = 0; h < 2; ++h) {
                            const float2 ia2 = half2of(ia4, h);
                            const float2 kb = fma2(ia2, make_float2(2.f, 2.f), make_float2(-1.f, -1.f));
                            out[h] = add2(u0[h], fma2(mul2(half2of(c24, h), ia2), q[h],
                                                      mul2(kb, sub2(u0[h], half2of(um4, h)))));
                        }
                        const float o[4] = {out[0].x, out[0].y, out[1].x, out[1].y};
                        if ((!QOUT || a.uout != nullptr) && colok && i < L.nzp) store4(up + fidx(L, i, j0), j0, L.nxp, o);
                        if (a.band != nullptr && sg.brow[r] != -1) {
                            float *bb = a.band + ((long long)ss * c.nt + a.n + 1) * L.nbandp;
                            if (sg.brow[r] >= 0) {
                                *reinterpret_cast<float4 *>(bb + sg.brow[r]) = make_float4(o[0], o[1], o[2], o[3]);
                            } else {
#pragma unroll
                                for (int p = 0; p < 4; ++p)
                                    if (in_band(L, i, j0 + p)) bb[band_index(L, i, j0 + p)] = o[p];
                            }
                        }
                    }
                    if (a.illum_utt) {
#pragma unroll
                        for (int h = 0; h < 2; ++h) {
                            const float2 d2 = add2(fma2(u0[h], make_float2(-2.f, -2.f), out[h]), half2of(um4, h));
                            acc_i[r][h] = fma2(d2, d2, acc_i[r][h]);
                        }
                    }
                }
                if (!a.illum_utt) {
                    acc_i[r][0] = fma2(u0[0], u0[0], acc_i[r][0]);
                    acc_i[r][1] = fma2(u0[1], u0[1], acc_i[r][1]);
                }
                if (WITH_H) {
                    // u(x+h) u(x-h); even h: points (0, 1) and (2, 3) on
                    // aligned lane pairs; odd h: (1, 2) paired, 0 and 3 scalar
#pragma unroll
                    for (int h = 0; h < NH; ++h) {
                        if ((h & 1) == 0) {
#pragma unroll
                            for (int q = 0; q < 2; ++q)
                                acc_h[h][q] = fma2(f2(w[WL + 2 * q + h], w[WL + 2 * q + 1 + h]),
                                                   f2(w[WL + 2 * q - h], w[WL + 2 * q + 1 - h]), acc_h[h][q]);
                        } else {
                            // odd h: points 1 and 2 on an aligned lane pair, 0 and 3 scalar
                            acc_h[h][0] = fma2(f2(w[WL + 1 + h], w[WL + 2 + h]), f2(w[WL + 1 - h], w[WL + 2 - h]),
                                               acc_h[h][0]);
                            acc_h[h][1].x = fmaf(w[WL + h], w[WL - h], acc_h[h][1].x);
                            acc_h[h][1].y = fmaf(w[WL + 3 + h], w[WL + 3 - h], acc_h[h][1].y);
                        }
                    }
                }
            }
        }
        if (threadIdx.x == 32) cp_async_wait_all(); // the slot staged in this iteration
        __syncthreads();
        if (s_abort) {
            abort_drain_ring<STAGES>(bars, s_desc, k, a0.c.status);
            return;
        }
    }
    if (cur_tile >= 0) flush();
}

// ----------------------------------------------------------- backward step
template <int RZ, int STAGES>
using BwdRing = Ring<8 * RZ, RADIUS, 2, 2, STAGES, 3 * 8 * RZ * TX * 4>; // + c2, injection, damping tiles

// The q tile of the extended operators: q = Lhat u + f delta_s of one halo
// tile on the TZ x (TX + 4 HE) columns bj - 2 HE .. bj + TX + 2 HE - 1 (the
// x-extension of the offsets 2h, |h| <= HE), zero where a column leaves the
// padded grid or a row its padded rows. The thread's own columns come from
// its registers (q_own_to_smem); the 2 HE columns on each side (q_edges_to_smem)
// as rows of 4 points (2 HE / 4 groups per side, TZ rows), which one warp
// computes with the paired Laplacian of the tile's own points (lap4: bitwise
// the same q).
template <int RZ, int HE, int TXS, int HX>
__device__ __forceinline__ void q_edges_to_smem(float *qs, const float *su, const ItemDesc &d, int bi, int bj,
                                                  const Lay2D &L, float src_scale)
{
    constexpr int TZ = 8 * RZ, QW = TX + 4 * HE, G = HE; // groups of 4 columns on each side: 2 HE / 4 * 2 = HE
    static_assert(HE % 2 == 0, "edge groups of 4 columns");
    constexpr int NU = TZ * G;                             // units of (row, group)
    const int wid = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (wid != 3) return;
    for (int u = lane; u < NU; u += 32) {
        const int r = u / G, g = u - r * G;
        const int c0 = g < G / 2 ? -2 * HE + 4 * g : TX + 4 * (g - G / 2); // first column of the group
        const float *ctr = su + (r + RADIUS) * TXS + HX + c0;
        float4 zc[1 + 2 * RADIUS];
#pragma unroll
        for (int kk = 0; kk < 1 + 2 * RADIUS; ++kk) zc[kk] = lds4(ctr + (kk - RADIUS) * TXS);
        const float4 a0 = lds4(ctr - 4), a2 = lds4(ctr + 4);
        const float4 a1 = zc[RADIUS];
        const float w[12] = {a0.x, a0.y, a0.z, a0.w, a1.x, a1.y, a1.z, a1.w, a2.x, a2.y, a2.z, a2.w};
        float2 q[2];
        lap4<4, 1 + 2 * RADIUS, false>(q, w, zc, 0);
        const float v[4] = {q[0].x, q[0].y, q[1].x, q[1].y};
        const int gi = bi + r;
        float qq[4];
#pragma unroll
        for (int p = 0; p < 4; ++p) {
            const int gj = bj + c0 + p;
            qq[p] = (gi < L.nzp && gj >= 0 && gj < L.nxp) ? v[p] : 0.f;
            if (gi == d.si && gj == d.sj) qq[p] += d.amp * src_scale;
        }
        *reinterpret_cast<float4 *>(qs + r * QW + c0 + 2 * HE) = make_float4(qq[0], qq[1], qq[2], qq[3]);
    }
}

template <int RZ, int HE>
__device__ __forceinline__ void q_own_to_smem(float *qs, const float2 (&q)[RZ][2], int i0, int j0, const Lay2D &L,
                                              int tx, int ty)
{
    constexpr int QW = TX + 4 * HE;
#pragma unroll
    for (int r = 0; r < RZ; ++r) {
        const bool rowok = i0 + r < L.nzp;
        // one 16-byte store per row (QW and 2 HE are multiples of 4)
        *reinterpret_cast<float4 *>(qs + (ty * RZ + r) * QW + 2 * HE + 4 * tx) =
            make_float4(rowok && j0 < L.nxp ? q[r][0].x : 0.f, rowok && j0 + 1 < L.nxp ? q[r][0].y : 0.f,
                        rowok && j0 + 2 < L.nxp ? q[r][1].x : 0.f, rowok && j0 + 3 < L.nxp ? q[r][1].y : 0.f);
    }
}

// Lhat of one halo tile at the thread's RZ x 4 points, in lane pairs
template <int RZ, int TXS, int HX>
__device__ __forceinline__ void tile_lap(float2 (&q)[RZ][2], const float *sf, int tx, int ty)
{
    float4 zc[RZ + 2 * RADIUS];
#pragma unroll
    for (int kk = 0; kk < RZ + 2 * RADIUS; ++kk) zc[kk] = lds4(&sf[(ty * RZ + kk) * TXS + HX + 4 * tx]);
#pragma unroll
    for (int r = 0; r < RZ; ++r) {
        const float *rw = &sf[(ty * RZ + r + RADIUS) * TXS + HX + 4 * tx];
        const float4 a0 = lds4(rw - 4), a2 = lds4(rw + 4);
        const float4 a1 = zc[r + RADIUS];
        const float w[12] = {a0.x, a0.y, a0.z, a0.w, a1.x, a1.y, a1.z, a1.w, a2.x, a2.y, a2.z, a2.w};
        lap4<4, RZ + 2 * RADIUS, false>(q[r], w, zc, r);
    }
}

template <int RZ>
__device__ __forceinline__ void add_source(float2 (&q)[RZ][2], int sslot, float amp)
{
#pragma unroll
    for (int r = 0; r < RZ; ++r) {
        if (sslot == r * 4 + 0) q[r][0].x += amp;
        if (sslot == r * 4 + 1) q[r][0].y += amp;
        if (sslot == r * 4 + 2) q[r][1].x += amp;
        if (sslot == r * 4 + 3) q[r][1].y += amp;
    }
}

// The q values a thread's row needs, columns 4 tx .. 4 tx + 4 HE + 3 of the
// q tile (x = y - 2 HE .. y + 2 HE + 1 for its 4 points y), as HE + 1
// 16-byte loads: lane pair j of them (columns 4 tx + 2j, 4 tx + 2j + 1) is
// half j & 1 of qv[j >> 1]
template <int HE>
__device__ __forceinline__ void q_row(float4 (&qv)[HE + 1], const float *qrow, int tx)
{
#pragma unroll
    for (int m = 0; m <= HE; ++m) qv[m] = lds4(qrow + 4 * tx + 4 * m);
}

// acc[lane][h + HE] += psi(y) q(y + 2h) for the two points of lane pair
// `lane` (points 2 lane, 2 lane + 1 of the thread's four) of one row
template <int HE>
__device__ __forceinline__ void ext_accumulate(float2 (&acc)[2][2 * HE + 1], float2 psi, int lane,
                                               const float4 (&qv)[HE + 1])
{
#pragma unroll
    for (int hh = 0; hh < 2 * HE + 1; ++hh) {
        const int j = lane + hh; // lane pair of columns y + 2h
        acc[lane][hh] = fma2(psi, half2of(qv[j >> 1], j & 1), acc[lane][hh]);
    }
}

// With extended imaging over offsets h = -HE..HE (Eq. 6): halo tiles wide
// enough for q^{m-1} on TX + 4 HE columns (x +- 2 HE), and that q row tile.
template <int RZ, int STAGES, int HE>
using BwdRingE = Ring<8 * RZ, RADIUS + 2 * HE, 2, 2, STAGES,
                      3 * 8 * RZ * TX * 4 + (HE > 0 ? 8 * RZ * (TX + 4 * HE) * 4 : 0)>;

// QIN: q^{m-1} is read as a point tile (into the first halo slot) instead of
// computed from a u^{m-1} halo tile (snapshot checkpoints, one model)
template <int RZ, int STAGES, int MINB, int NM, int HE = 0, bool QIN = false>
__global__ void __launch_bounds__(TPB, MINB) k_bwd_step(const __grid_constant__ Batch<BwdArgs, NM> B)
{
    static_assert(!QIN || (HE == 0 && NM == 1), "q input: plain backward step of one model");
    static_assert(HE == 0 || (HE % 2 == 0 && NM == 1), "extended imaging: even HE, one model");
    using R = BwdRingE<RZ, STAGES, HE>;
    constexpr int TZ = 8 * RZ;
    constexpr int HX = RADIUS + 2 * HE;   // a multiple of 4: TMA x offsets stay 16-byte aligned
    constexpr int NE = 2 * HE + 1;        // extended offsets
    constexpr int QW = TX + 4 * HE;       // columns of the q tile
    constexpr int TXS = R::TXS;
    constexpr int D = STAGES - 1;
    // item j's descriptor is staged (lane 0 of warp 1) in iteration j-D-1
    // and read in iteration j-D (copy issue) and j-1 (prefetch) and j: always
    // at least one barrier after it was written, for any D >= 1
    static_assert(D >= 1 && D + 2 <= DESC_RING, "needs 2 <= STAGES <= 7");
    // live descriptor slots in iteration k: k .. k+D+1 (read, issued, staged)
    extern __shared__ unsigned char smem_raw[];
    __shared__ int s_abort;
    __shared__ ItemDesc s_desc[DESC_RING];
    unsigned char *smem = align_smem(smem_raw);
    uint64_t *bars = reinterpret_cast<uint64_t *>(smem);
    float *c2s = reinterpret_cast<float *>(R::extra(smem));
    float *sinj = c2s + TZ * TX;
    float *dms = sinj + TZ * TX; // damping tile (sponge tiles)
    float *qs = dms + TZ * TX;   // q^{m-1} on columns bj - 2 HE .. bj + TX + 2 HE - 1 (HE > 0)
    (void)qs;

    // launch-wide values (time level, mode) are those of model 0
    const BwdArgs &a0 = B.m[0];
    const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
    const int m = a0.m;
    const bool recon = a0.recon != 0;
    const bool need_band = recon && m >= 3; // u^{m-2} in the sponge comes from checkpoint m-2 >= 1

    if (threadIdx.x == 0) {
        for (int k = 0; k < STAGES; ++k) mbar_init(smem_u32(&bars[k]), 1);
        fence_mbar_init();
        s_abort = 0;
    }
    for (int e = threadIdx.x; e < TZ * TX; e += TPB) sinj[e] = 0.f;
    __syncthreads();

    __shared__ Cursor s_cu;
    auto stage = [&](int slot) { stage_desc_async<1>(&s_desc[slot % DESC_RING], s_cu, B, m - 1, true); };
    auto issue = [&](const ItemDesc &d, int k) {
        const BwdArgs &a = B.m[NM == 1 ? 0 : d.model];
        const int bz = d.tile / a.c.ntx, bx = d.tile - bz * a.c.ntx;
        const int bi = bz * TZ, bj = bx * TX;
        const int st = k % STAGES;
        const uint32_t bar = smem_u32(&bars[st]);
        const bool need_ua = !QIN && recon && m >= 2;
        fence_proxy_async_smem();
        mbar_expect_tx(bar, ((QIN ? 1 : 2) * R::HALO + (need_ua ? 2 : 1) * R::PT + (QIN ? R::PT : 0)) * 4);
        if constexpr (QIN)
            tma_load_3d(smem_u32(R::halo(smem, st, 0)), &a.tm_ub, GXL + bj, bi + GZ, d.s, bar);
        else
            tma_load_3d(smem_u32(R::halo(smem, st, 0)), &a.tm_ub, GXL + bj - HX, bi, d.s, bar);
        tma_load_3d(smem_u32(R::halo(smem, st, 1)), &a.tm_pa, GXL + bj - HX, bi, d.s, bar);
        tma_load_3d(smem_u32(R::point(smem, st, 1)), &a.tm_pb, GXL + bj, bi + GZ, d.s, bar);
        if (need_ua) tma_load_3d(smem_u32(R::point(smem, st, 0)), &a.tm_ua, GXL + bj, bi + GZ, d.s, bar);
    };
    // lane 0 of warp 1 walks the chunks and stages descriptors; thread 0
    // issues the copies of a descriptor staged one barrier earlier
    if (threadIdx.x == 32) {
        cursor_init(s_cu, B);
        for (int k = 0; k <= D; ++k) stage(k);
        cp_async_wait_all();
    }
    __syncthreads();
    if (threadIdx.x == 0)
        for (int k = 0; k < D; ++k)
            if (s_desc[k].tile >= 0) issue(s_desc[k], k);

    float2 acc_g[RZ][2];
    float2 acc_e[RZ][2][NE]; // extended image at (own point y, h): sum psi^m(y) q^{m-1}(y + 2h)
    int cur_tile = -1, cur_model = 0, bi = 0, bj = 0, i0 = 0, j0 = 0;
    bool tile_sponge = false, colok = false;
    SpongeInfo<RZ> sg;

    // gradient accumulators of the current tile to global memory
    auto flush = [&]() {
        const BwdArgs &a = B.m[NM == 1 ? 0 : cur_model];
        const Lay2D &L = a.c.L;
#pragma unroll
        for (int r = 0; r < RZ; ++r) {
            const int i = i0 + r;
            if ((L.nxp & 3) == 0 && i < L.nzp && j0 + 3 < L.nxp) {
                // the thread's 4 columns: one vector reduction per sum
                red_add4(a.acc_grad + (long long)i * L.nxp + j0, acc_g[r][0].x, acc_g[r][0].y, acc_g[r][1].x,
                         acc_g[r][1].y);
                if constexpr (HE > 0) {
#pragma unroll
                    for (int e = 0; e < NE; ++e)
                        red_add4(a.acc_ext + ((long long)e * L.nzp + i) * L.nxp + j0, acc_e[r][0][e].x, acc_e[r][0][e].y,
                                 acc_e[r][1][e].x, acc_e[r][1][e].y);
                }
                continue;
            }
#pragma unroll
            for (int p = 0; p < 4; ++p) {
                const int j = j0 + p;
                const float v = p < 2 ? (p == 0 ? acc_g[r][0].x : acc_g[r][0].y) : (p == 2 ? acc_g[r][1].x : acc_g[r][1].y);
                if (i < L.nzp && j < L.nxp) atomicAdd(a.acc_grad + (long long)i * L.nxp + j, v);
                if constexpr (HE > 0) {
                    if (i < L.nzp && j < L.nxp)
#pragma unroll
                        for (int e = 0; e < NE; ++e)
                            atomicAdd(a.acc_ext + ((long long)e * L.nzp + i) * L.nxp + j, (p & 1) ? acc_e[r][p >> 1][e].y : acc_e[r][p >> 1][e].x);
                }
            }
        }
    };

    // adjoint-source entry of this thread for an item (one entry per thread
    // is prefetched; further entries of a crowded tile are read late)
    auto fetch_adj = [&](const ItemDesc &v, int &loc, float &val) {
        loc = -1;
        val = 0.f;
        const int e = v.rb + (int)threadIdx.x;
        if (v.tile >= 0 && e < v.re) {
            const BwdArgs &a = B.m[NM == 1 ? 0 : v.model];
            loc = a.rt.ent[e].x;
            val = a.adj[(long long)m * a.nent + e] * a.adj_scale;
        }
    };

    // checkpointed sponge values of u^{m-2} of one item of the current tile
    auto fetch_band = [&](int s, float4 (&bv)[RZ]) {
        const BwdArgs &a = B.m[NM == 1 ? 0 : cur_model];
        const StepCommon &c = a.c;
        const Lay2D &L = c.L;
#pragma unroll
        for (int r = 0; r < RZ; ++r) {
            bv[r] = make_float4(0.f, 0.f, 0.f, 0.f);
            if (need_band && sg.brow[r] != -1) {
                const float *bb = a.band + ((long long)s * c.nt + (m - 2)) * L.nbandp;
                if (sg.brow[r] >= 0) {
                    bv[r] = __ldcs(reinterpret_cast<const float4 *>(bb + sg.brow[r]));
                } else {
                    const int i = i0 + r;
                    float t[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
                    for (int p = 0; p < 4; ++p)
                        if (in_band(L, i, j0 + p)) t[p] = __ldcs(bb + band_index(L, i, j0 + p));
                    bv[r] = make_float4(t[0], t[1], t[2], t[3]);
                }
            }
        }
    };

    int adj_loc;
    float adj_val;
    fetch_adj(s_desc[0], adj_loc, adj_val);
    float4 bval[RZ];
    bool bval_ok = false; // bval holds the current item's checkpoint values
    int k = 0;
    for (;; ++k) {
        if (threadIdx.x == 0) {
            const ItemDesc d = s_desc[(k + D) % DESC_RING];
            if (d.tile >= 0) issue(d, k + D);
        } else if (threadIdx.x == 32) {
            stage(k + D + 1);
        }
        const ItemDesc now = s_desc[k % DESC_RING];
        if (now.tile < 0) {
            if (threadIdx.x == 32) cp_async_wait_all(); // (none in flight once the cursor is done)
            break;
        }
        const ItemDesc nx = s_desc[(k + 1) % DESC_RING];
        const int s = now.s;
        const int mi = NM == 1 ? 0 : now.model;
        const BwdArgs &a = B.m[mi];
        const StepCommon &c = a.c;
        const Lay2D &L = c.L;
        if (now.tile != cur_tile || mi != cur_model) {
            if (cur_tile >= 0) flush();
            cur_tile = now.tile;
            cur_model = mi;
            const int bz = cur_tile / c.ntx, bx = cur_tile - bz * c.ntx;
            bi = bz * TZ;
            bj = bx * TX;
            i0 = bi + ty * RZ;
            j0 = bj + 4 * tx;
            tile_sponge = bi < L.P || bi + TZ > L.P + L.nz || bj < L.P || bj + TX > L.P + L.nx;
            colok = j0 < L.nxp;
            if (tile_sponge) sg.init(L, i0, j0);
#pragma unroll
            for (int r = 0; r < RZ; ++r) acc_g[r][0] = acc_g[r][1] = make_float2(0.f, 0.f);
            if constexpr (HE > 0) {
#pragma unroll
                for (int r = 0; r < RZ; ++r)
#pragma unroll
                    for (int p = 0; p < 2; ++p)
#pragma unroll
                        for (int e = 0; e < NE; ++e) acc_e[r][p][e] = make_float2(0.f, 0.f);
            }
            load_coef_tiles<TZ>(c2s, dms, c, tile_sponge, bi, bj);
            bval_ok = false;
            __syncthreads();
        }
        float4 bnow[RZ];
        if (tile_sponge) {
            if (!bval_ok) fetch_band(s, bval);
#pragma unroll
            for (int r = 0; r < RZ; ++r) bnow[r] = bval[r];
        }
        const bool has_rec = now.rb < now.re; // uniform over the CTA
        const int my_loc = adj_loc;
        if (has_rec) {
            if (adj_loc >= 0) atomicAdd(&sinj[adj_loc], adj_val);
            for (int e = now.rb + TPB + (int)threadIdx.x; e < now.re; e += TPB)
                atomicAdd(&sinj[a.rt.ent[e].x], a.adj[(long long)m * a.nent + e] * a.adj_scale);
        }
        // prefetch for the next item: adjoint entry, and its checkpoint values
        // when it is on the same tile
        if (nx.re > nx.rb) {
            fetch_adj(nx, adj_loc, adj_val);
        } else { // (warp-uniform) no receivers in the next item's tile
            adj_loc = -1;
            adj_val = 0.f;
        }
        bval_ok = tile_sponge && nx.tile == cur_tile && (NM == 1 || nx.model == cur_model);
        if (bval_ok) fetch_band(nx.s, bval);
        if (has_rec) __syncthreads();
        const int st = k % STAGES;
        const bool ready = stage_ready<STAGES>(bars, k, &s_abort);
        const float *su = R::halo(smem, st, 0);
        const float *sp = R::halo(smem, st, 1);
        float2 qu[RZ][2], qp[RZ][2];
        if constexpr (HE > 0) {
            // q^{m-1} on the tile and 2 HE columns on each side (zero outside
            // the padded grid), for the extended image
            if (ready) {
                tile_lap<RZ, TXS, HX>(qu, su, tx, ty);
                if ((unsigned)(now.si - bi) < (unsigned)TZ && (unsigned)(now.sj - bj) < (unsigned)TX)
                    add_source<RZ>(qu, source_slot<RZ>(now, i0, j0), now.amp * c.src_scale);
                q_own_to_smem<RZ, HE>(qs, qu, i0, j0, L, tx, ty);
                q_edges_to_smem<RZ, HE, TXS, HX>(qs, su, now, bi, bj, L, c.src_scale);
            }
            __syncthreads();
        }
        if (ready) {
            const float *pua = R::point(smem, st, 0);
            const float *ppb = R::point(smem, st, 1);
            const long long so = (long long)s * L.fstride;
            // the shot's source cell, if it lies in this tile (warp-uniform)
            const bool src_tile = (unsigned)(now.si - bi) < (unsigned)TZ && (unsigned)(now.sj - bj) < (unsigned)TX;
            const int sslot = src_tile ? source_slot<RZ>(now, i0, j0) : -1;

            // q^{m-1} = Lhat u^{m-1} + f(t_{m-1}) delta_s (as in the forward
            // step m-1; done above with the extended image), then Lhat psi^{m+1};
            // one column window live at a time
#pragma unroll
            for (int fld = (HE > 0 || QIN) ? 1 : 0; fld < 2; ++fld) {
                const float *sf = fld == 0 ? su : sp;
                float4 zc[RZ + 2 * RADIUS];
#pragma unroll
                for (int kk = 0; kk < RZ + 2 * RADIUS; ++kk) zc[kk] = lds4(&sf[(ty * RZ + kk) * TXS + HX + 4 * tx]);
#pragma unroll
                for (int r = 0; r < RZ; ++r) {
                    const float *rw = &sf[(ty * RZ + r + RADIUS) * TXS + HX + 4 * tx];
                    const float4 a0 = lds4(rw - 4), a2 = lds4(rw + 4);
                    const float4 a1 = zc[r + RADIUS];
                    const float w[12] = {a0.x, a0.y, a0.z, a0.w, a1.x, a1.y, a1.z, a1.w, a2.x, a2.y, a2.z, a2.w};
                    if (fld == 0)
                        lap4<4, RZ + 2 * RADIUS, false>(qu[r], w, zc, r);
                    else
                        lap4<4, RZ + 2 * RADIUS, false>(qp[r], w, zc, r);
                }
            }
#pragma unroll
            for (int r = 0; r < RZ; ++r) {
                const float amp = now.amp * c.src_scale;
                if constexpr (QIN) { // the kept q^{m-1}, its source term included
                    const float4 q4 = lds4(&su[(ty * RZ + r) * TX + 4 * tx]);
                    qu[r][0] = lo2(q4);
                    qu[r][1] = hi2(q4);
                } else if (HE == 0 && src_tile) {
                    if (sslot == r * 4 + 0) qu[r][0].x += amp;
                    if (sslot == r * 4 + 1) qu[r][0].y += amp;
                    if (sslot == r * 4 + 2) qu[r][1].x += amp;
                    if (sslot == r * 4 + 3) qu[r][1].y += amp;
                }
                if (has_rec) {
                    const float4 inj = lds4(&sinj[(ty * RZ + r) * TX + 4 * tx]);
                    qp[r][0] = add2(qp[r][0], lo2(inj));
                    qp[r][1] = add2(qp[r][1], hi2(inj));
                }
                const int sr = ty * RZ + r + RADIUS;
                const float4 uc = QIN ? make_float4(0.f, 0.f, 0.f, 0.f) : lds4(&su[sr * TXS + HX + 4 * tx]); // (QIN: no rebuild)
                const float4 pc = lds4(&sp[sr * TXS + HX + 4 * tx]);
                const float2 p1[2] = {lo2(pc), hi2(pc)};
                const float2 u1[2] = {lo2(uc), hi2(uc)};
                const float4 ua4 = lds4(&pua[(ty * RZ + r) * TX + 4 * tx]);
                const float4 pb4 = lds4(&ppb[(ty * RZ + r) * TX + 4 * tx]);
                const float4 c24 = lds4(&c2s[(ty * RZ + r) * TX + 4 * tx]);
                float4 qv[HE + 1]; // HE > 0: the row's q values for the extended image
                if constexpr (HE > 0) q_row<HE>(qv, qs + (ty * RZ + r) * QW, tx);
                if (!tile_sponge) {
                    float2 pn[2], un[2];
#pragma unroll
                    for (int h = 0; h < 2; ++h) {
                        const float2 c2v = half2of(c24, h);
                        pn[h] = add2(p1[h], fma2(c2v, qp[r][h], sub2(p1[h], half2of(pb4, h))));
                        acc_g[r][h] = fma2(pn[h], qu[r][h], acc_g[r][h]);
                        if constexpr (HE > 0) ext_accumulate<HE>(acc_e[r], pn[h], h, qv);
                        // leap_back on two lanes: u1 - (-(c2 q) + (u^m - u1))
                        un[h] = sub2(u1[h], fma2(make_float2(-c2v.x, -c2v.y), qu[r][h], sub2(half2of(ua4, h), u1[h])));
                    }
                    *reinterpret_cast<float4 *>(a.pb + so + fidx(L, i0 + r, j0)) =
                        make_float4(pn[0].x, pn[0].y, pn[1].x, pn[1].y);
                    if (recon && m >= 2)
                        *reinterpret_cast<float4 *>(a.ua + so + fidx(L, i0 + r, j0)) =
                            make_float4(un[0].x, un[0].y, un[1].x, un[1].y);
                } else {
                    // damped adjoint update (identical to the plain one where
                    // eta = 0); sponge values of u^{m-2} from the checkpoint
                    const int i = i0 + r;
                    const float4 ia4 = lds4(&dms[(ty * RZ + r) * TX + 4 * tx]);
                    float2 pn[2], un[2];
#pragma unroll
                    for (int h = 0; h < 2; ++h) {
                        const float2 ia2 = half2of(ia4, h);
                        const float2 c2v = half2of(c24, h);
                        const float2 kb = fma2(ia2, make_float2(2.f, 2.f), make_float2(-1.f, -1.f));
                        pn[h] = add2(p1[h], fma2(mul2(c2v, ia2), qp[r][h], mul2(kb, sub2(p1[h], half2of(pb4, h)))));
                        acc_g[r][h] = fma2(pn[h], qu[r][h], acc_g[r][h]);
                        if constexpr (HE > 0) ext_accumulate<HE>(acc_e[r], pn[h], h, qv);
                        un[h] = sub2(u1[h], fma2(make_float2(-c2v.x, -c2v.y), qu[r][h], sub2(half2of(ua4, h), u1[h])));
                    }
                    float pnew[4] = {pn[0].x, pn[0].y, pn[1].x, pn[1].y};
                    float unew[4] = {un[0].x, un[0].y, un[1].x, un[1].y};
                    if (sg.brow[r] >= 0) {
                        unew[0] = bnow[r].x; unew[1] = bnow[r].y; unew[2] = bnow[r].z; unew[3] = bnow[r].w;
                    } else if (sg.brow[r] == -2) {
#pragma unroll
                        for (int p = 0; p < 4; ++p)
                            if (in_band(L, i, j0 + p)) unew[p] = comp(bnow[r], p);
                    }
                    if (colok && i < L.nzp) {
                        store4(a.pb + so + fidx(L, i, j0), j0, L.nxp, pnew);
                        if (recon && m >= 2) store4(a.ua + so + fidx(L, i, j0), j0, L.nxp, unew);
                    }
                }
            }
        }
        if (threadIdx.x == 32) cp_async_wait_all(); // the slot staged in this iteration
        __syncthreads();
        if (s_abort) {
            abort_drain_ring<STAGES>(bars, s_desc, k, a0.c.status);
            return;
        }
        if (has_rec) {
            if (my_loc >= 0) sinj[my_loc] = 0.f;
            for (int e = now.rb + TPB + (int)threadIdx.x; e < now.re; e += TPB) sinj[a.rt.ent[e].x] = 0.f;
            __syncthreads();
        }
    }
    if (cur_tile >= 0) flush();
}

// -------------------------------------------------------------- Born step
// The tangent-linear of the forward step along dv (Born modelling, Eq. 4, in
// the discrete form whose adjoint is the backward step):
//   u^{n+1}  = u^n  + fma(c2 ia, q^n, kb (u^n - u^{n-1})),      q^n = Lhat u^n + f delta_s
//   du^{n+1} = du^n + ia (c2 Lhat du^n + dc2 q^n) + kb (du^n - du^{n-1}),
// dc2 = 2 c2 dv / v, ia = 1 / (1 + eta dt), kb = 2 ia - 1; Born traces du^n at
// the receivers. Same tiles, ring and scheduling as the backward step (two
// halo fields and two point fields per item).
template <int RZ, int STAGES>
using BornRing = Ring<8 * RZ, RADIUS, 2, 2, STAGES, 3 * 8 * RZ * TX * 4>; // + c2, dc2, damping tiles

// Extended Born (Eq. 5, offsets h = -HE..HE): wider halo tiles for q on
// TX + 4 HE columns, plus the 2 HE + 1 planes of D~(y, h) and the q tile.
template <int RZ, int STAGES, int HE>
using BornRingE = Ring<8 * RZ, RADIUS + 2 * HE, 2, 2, STAGES,
                       2 * 8 * RZ * TX * 4 + (HE > 0 ? (2 * HE + 1) * 8 * RZ * TX * 4 + 8 * RZ * (TX + 4 * HE) * 4 : 0)>;

template <int RZ, int STAGES, int MINB, int HE = 0>
__global__ void __launch_bounds__(TPB, MINB) k_born_step(const __grid_constant__ Batch<BornArgs, 1> B)
{
    static_assert(HE % 2 == 0, "extended Born: even HE (16-byte aligned TMA x offsets)");
    using R = BornRingE<RZ, STAGES, HE>;
    constexpr int TZ = 8 * RZ;
    constexpr int HX = RADIUS + 2 * HE;
    constexpr int NE = 2 * HE + 1;
    constexpr int QW = TX + 4 * HE;
    constexpr int TXS = R::TXS;
    constexpr int D = STAGES - 1;
    static_assert(D >= 1 && D + 2 <= DESC_RING, "needs 2 <= STAGES <= 7");
    extern __shared__ unsigned char smem_raw[];
    __shared__ int s_abort;
    __shared__ ItemDesc s_desc[DESC_RING];
    __shared__ Cursor s_cu;
    unsigned char *smem = align_smem(smem_raw);
    uint64_t *bars = reinterpret_cast<uint64_t *>(smem);
    float *c2s = reinterpret_cast<float *>(R::extra(smem));
    float *dms = c2s + TZ * TX;  // damping tile (sponge tiles); dc2 is read per point from L2
    float *des = dms + TZ * TX;  // HE > 0: planes D~(y, h), h = -HE..HE
    float *qs = des + NE * TZ * TX; // HE > 0: q^n on columns bj - 2 HE .. bj + TX + 2 HE - 1
    (void)qs;
    (void)QW;

    const BornArgs &a = B.m[0];
    const StepCommon &c = a.c;
    const Lay2D &L = c.L;
    const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;

    if (threadIdx.x == 0) {
        for (int k = 0; k < STAGES; ++k) mbar_init(smem_u32(&bars[k]), 1);
        fence_mbar_init();
        s_abort = 0;
    }
    __syncthreads();

    auto stage = [&](int slot) { stage_desc_async<1>(&s_desc[slot % DESC_RING], s_cu, B, a.n, !a.last); };
    auto issue = [&](const ItemDesc &d, int k) {
        const int bz = d.tile / c.ntx, bx = d.tile - bz * c.ntx;
        const int bi = bz * TZ, bj = bx * TX;
        const int st = k % STAGES;
        const uint32_t bar = smem_u32(&bars[st]);
        fence_proxy_async_smem();
        mbar_expect_tx(bar, (2 * R::HALO + (a.last ? 0 : 2 * R::PT)) * 4);
        tma_load_3d(smem_u32(R::halo(smem, st, 0)), &a.tm_u, GXL + bj - HX, bi, d.s, bar);
        tma_load_3d(smem_u32(R::halo(smem, st, 1)), &a.tm_du, GXL + bj - HX, bi, d.s, bar);
        if (!a.last) {
            tma_load_3d(smem_u32(R::point(smem, st, 0)), &a.tm_up, GXL + bj, bi + GZ, d.s, bar);
            tma_load_3d(smem_u32(R::point(smem, st, 1)), &a.tm_dup, GXL + bj, bi + GZ, d.s, bar);
        }
    };
    if (threadIdx.x == 32) {
        cursor_init(s_cu, B);
        for (int k = 0; k <= D; ++k) stage(k);
        cp_async_wait_all();
    }
    __syncthreads();
    if (threadIdx.x == 0)
        for (int k = 0; k < D; ++k)
            if (s_desc[k].tile >= 0) issue(s_desc[k], k);

    int cur_tile = -1, bi = 0, bj = 0, i0 = 0, j0 = 0;
    bool tile_sponge = false, colok = false;
    SpongeInfo<RZ> sg;
    for (int k = 0;; ++k) {
        if (threadIdx.x == 0) {
            const ItemDesc d = s_desc[(k + D) % DESC_RING];
            if (d.tile >= 0) issue(d, k + D);
        } else if (threadIdx.x == 32) {
            stage(k + D + 1);
        }
        const ItemDesc now = s_desc[k % DESC_RING];
        if (now.tile < 0) {
            if (threadIdx.x == 32) cp_async_wait_all();
            break;
        }
        const int s = now.s;
        if (now.tile != cur_tile) {
            cur_tile = now.tile;
            const int bz = cur_tile / c.ntx, bx = cur_tile - bz * c.ntx;
            bi = bz * TZ;
            bj = bx * TX;
            i0 = bi + ty * RZ;
            j0 = bj + 4 * tx;
            tile_sponge = bi < L.P || bi + TZ > L.P + L.nz || bj < L.P || bj + TX > L.P + L.nx;
            colok = j0 < L.nxp;
            if (tile_sponge) sg.init(L, i0, j0);
            if constexpr (HE > 0) {
                // c2, damping and the 2 HE + 1 planes of D~
                float *dst[NE + 2];
                const float *src[NE + 2];
                dst[0] = c2s;
                src[0] = c.c2;
                dst[1] = dms;
                src[1] = tile_sponge ? c.damp : nullptr;
#pragma unroll
                for (int e = 0; e < NE; ++e) {
                    dst[2 + e] = des + e * TZ * TX;
                    src[2 + e] = a.dext + e * L.fstride;
                }
                load_tiles<TZ, NE + 2>(dst, src, L, bi, bj);
            } else {
                load_coef_tiles<TZ>(c2s, dms, c, tile_sponge, bi, bj);
            }
            __syncthreads();
        }
        const int st = k % STAGES;
        const bool ready = stage_ready<STAGES>(bars, k, &s_abort);
        float2 qu[RZ][2];
        if constexpr (HE > 0) {
            // q^n on the tile and 2 HE columns on each side, for the
            // extended scattering source
            if (ready && !a.last) {
                const float *su = R::halo(smem, st, 0);
                tile_lap<RZ, TXS, HX>(qu, su, tx, ty);
                if ((unsigned)(now.si - bi) < (unsigned)TZ && (unsigned)(now.sj - bj) < (unsigned)TX)
                    add_source<RZ>(qu, source_slot<RZ>(now, i0, j0), now.amp * c.src_scale);
                q_own_to_smem<RZ, HE>(qs, qu, i0, j0, L, tx, ty);
                q_edges_to_smem<RZ, HE, TXS, HX>(qs, su, now, bi, bj, L, c.src_scale);
            }
            __syncthreads();
        }
        if (ready) {
            const float *su = R::halo(smem, st, 0);
            const float *sd = R::halo(smem, st, 1);
            // Born traces du^n = R du^n (one warp-uniform test skips the
            // tiles without receivers)
            if (now.re > now.rb) {
                float *ds = a.dseis + ((long long)s * c.nt + a.n) * c.nrec;
#pragma unroll 1
                for (int e = now.rb + (int)threadIdx.x; e < now.re; e += TPB) {
                    const int2 en = a.rt.ent[e];
                    const int zl = en.x / TX, xl = en.x - zl * TX;
                    ds[en.y] = sd[(zl + RADIUS) * TXS + HX + xl];
                }
            }
            if (!a.last) {
                const float *pu = R::point(smem, st, 0);
                const float *pd = R::point(smem, st, 1);
                const long long so = (long long)s * L.fstride;
                // the shot's source cell, if it lies in this tile (warp-uniform)
                const bool src_tile = (unsigned)(now.si - bi) < (unsigned)TZ && (unsigned)(now.sj - bj) < (unsigned)TX;
                const int sslot = src_tile ? source_slot<RZ>(now, i0, j0) : -1;
                // dc2 of the thread's points, one float4 per row from L2
                // (the tile stays out of shared memory: four CTAs per SM)
                float4 dcg[RZ];
#pragma unroll
                for (int r = 0; r < RZ; ++r)
                    dcg[r] = (HE == 0 && i0 + r < L.nzp)
                                 ? __ldg(reinterpret_cast<const float4 *>(a.dc2 + fidx(L, i0 + r, j0)))
                                 : make_float4(0.f, 0.f, 0.f, 0.f);
                float2 qd[RZ][2];
#pragma unroll
                for (int fld = HE > 0 ? 1 : 0; fld < 2; ++fld) {
                    const float *sf = fld == 0 ? su : sd;
                    float4 zc[RZ + 2 * RADIUS];
#pragma unroll
                    for (int kk = 0; kk < RZ + 2 * RADIUS; ++kk) zc[kk] = lds4(&sf[(ty * RZ + kk) * TXS + HX + 4 * tx]);
#pragma unroll
                    for (int r = 0; r < RZ; ++r) {
                        const float *rw = &sf[(ty * RZ + r + RADIUS) * TXS + HX + 4 * tx];
                        const float4 a0 = lds4(rw - 4), a2 = lds4(rw + 4);
                        const float4 a1 = zc[r + RADIUS];
                        const float w[12] = {a0.x, a0.y, a0.z, a0.w, a1.x, a1.y, a1.z, a1.w, a2.x, a2.y, a2.z, a2.w};
                        if (fld == 0)
                            lap4<4, RZ + 2 * RADIUS, false>(qu[r], w, zc, r);
                        else
                            lap4<4, RZ + 2 * RADIUS, false>(qd[r], w, zc, r);
                    }
                }
                const float amp = now.amp * c.src_scale;
#pragma unroll
                for (int r = 0; r < RZ; ++r) {
                    if (HE == 0 && src_tile) {
                        if (sslot == r * 4 + 0) qu[r][0].x += amp;
                        if (sslot == r * 4 + 1) qu[r][0].y += amp;
                        if (sslot == r * 4 + 2) qu[r][1].x += amp;
                        if (sslot == r * 4 + 3) qu[r][1].y += amp;
                    }
                    const int sr = ty * RZ + r + RADIUS;
                    const float4 uc = lds4(&su[sr * TXS + HX + 4 * tx]);
                    const float4 dc = lds4(&sd[sr * TXS + HX + 4 * tx]);
                    const float4 up4 = lds4(&pu[(ty * RZ + r) * TX + 4 * tx]);
                    const float4 dp4 = lds4(&pd[(ty * RZ + r) * TX + 4 * tx]);
                    const float4 c24 = lds4(&c2s[(ty * RZ + r) * TX + 4 * tx]);
                    const float4 dc24 = dcg[r];
                    // extended scattering source S(y) = sum_h D~(y, h) q(y + 2h)
                    float2 sx[2] = {make_float2(0.f, 0.f), make_float2(0.f, 0.f)};
                    if constexpr (HE > 0) {
                        float4 qv[HE + 1];
                        q_row<HE>(qv, qs + (ty * RZ + r) * QW, tx);
#pragma unroll
                        for (int hh = 0; hh < NE; ++hh) {
                            const float4 d4 = lds4(&des[(hh * TZ + ty * RZ + r) * TX + 4 * tx]);
                            // lane pairs hh and hh + 1: columns y + 2h of points (0, 1) and (2, 3)
                            sx[0] = fma2(lo2(d4), half2of(qv[hh >> 1], hh & 1), sx[0]);
                            sx[1] = fma2(hi2(d4), half2of(qv[(hh + 1) >> 1], (hh + 1) & 1), sx[1]);
                        }
                    }
                    float2 un[2], dn[2];
                    if (!tile_sponge) {
#pragma unroll
                        for (int h = 0; h < 2; ++h) {
                            const float2 u1 = half2of(uc, h), d1 = half2of(dc, h);
                            un[h] = add2(u1, fma2(half2of(c24, h), qu[r][h], sub2(u1, half2of(up4, h))));
                            if constexpr (HE > 0)
                                dn[h] = add2(d1, fma2(half2of(c24, h), qd[r][h], add2(sx[h], sub2(d1, half2of(dp4, h)))));
                            else
                                dn[h] = add2(d1, fma2(half2of(c24, h), qd[r][h],
                                                      fma2(half2of(dc24, h), qu[r][h], sub2(d1, half2of(dp4, h)))));
                        }
                    } else {
                        const float4 ia4 = lds4(&dms[(ty * RZ + r) * TX + 4 * tx]);
#pragma unroll
                        for (int h = 0; h < 2; ++h) {
                            const float2 ia2 = half2of(ia4, h);
                            const float2 kb = fma2(ia2, make_float2(2.f, 2.f), make_float2(-1.f, -1.f));
                            const float2 u1 = half2of(uc, h), d1 = half2of(dc, h);
                            un[h] = add2(u1, fma2(mul2(half2of(c24, h), ia2), qu[r][h], mul2(kb, sub2(u1, half2of(up4, h)))));
                            const float2 src2 = HE > 0 ? fma2(half2of(c24, h), qd[r][h], sx[h])
                                                       : fma2(half2of(c24, h), qd[r][h], mul2(half2of(dc24, h), qu[r][h]));
                            dn[h] = add2(d1, fma2(ia2, src2, mul2(kb, sub2(d1, half2of(dp4, h)))));
                        }
                    }
                    const int i = i0 + r;
                    if (colok && i < L.nzp) {
                        const float uo[4] = {un[0].x, un[0].y, un[1].x, un[1].y};
                        const float dox[4] = {dn[0].x, dn[0].y, dn[1].x, dn[1].y};
                        store4(a.uout + so + fidx(L, i, j0), j0, L.nxp, uo);
                        store4(a.duout + so + fidx(L, i, j0), j0, L.nxp, dox);
                        if (tile_sponge && a.band != nullptr && sg.brow[r] != -1) {
                            float *bb = a.band + ((long long)s * c.nt + a.n + 1) * L.nbandp;
                            if (sg.brow[r] >= 0) {
                                *reinterpret_cast<float4 *>(bb + sg.brow[r]) = make_float4(uo[0], uo[1], uo[2], uo[3]);
                            } else {
#pragma unroll
                                for (int p = 0; p < 4; ++p)
                                    if (in_band(L, i, j0 + p)) bb[band_index(L, i, j0 + p)] = uo[p];
                            }
                        }
                    }
                }
            }
        }
        if (threadIdx.x == 32) cp_async_wait_all();
        __syncthreads();
        if (s_abort) {
            abort_drain_ring<STAGES>(bars, s_desc, k, c.status);
            return;
        }
    }
}

// ------------------------------------ offset Hessian beside the plain step
// The offset-Hessian diagonal of one time level as a kernel of its own
// (Sec. 3): acc_offh[h][x] += sum_s u_s^n(x + h e_x) u_s^n(x - h e_x),
// h = 0..hmax, at the physical points (u = 0 outside the padded grid: the
// ghost columns), launched after the plain forward step of the level (the
// split offset-Hessian variants). A CTA takes one 64 x 8 tile of the physical
// region and a chunk of shots; the tile's rows with 12 columns on each side
// come through a shared-memory ring of cp.async copies, SPS shots per stage
// (one barrier per stage); each thread sums the products of its 4 points of
// one row in registers across the chunk, two shots at a time (both windows
// read before the products), and adds them with one vector reduction per
// offset.
__device__ __forceinline__ void cp_async16(void *dst, const void *src)
{
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(smem_u32(dst)), "l"(src) : "memory");
}

template <int NHC, int NST, int SPS>
__global__ void __launch_bounds__(TPB, 4) k_offh_level(const float *__restrict__ u, const Lay2D L, int ns,
                                                       int chunk, int hmax, float *acc_offh)
{
    constexpr int WL = HMAX_LIMIT, NW = (2 * WL + 4) / 4;
    constexpr int RW = TX + 2 * WL;   // a staged row: physical columns ixb - WL .. ixb + TX + WL - 1
    constexpr int NCH = 8 * (RW / 4); // 16-byte pieces of one shot's rows
    static_assert(NCH <= 2 * TPB, "two pieces per thread");
    __shared__ __align__(16) float sm[NST][SPS][8 * RW];
    const int ntz = (L.nz + 7) / 8, ntx = (L.nx + TX - 1) / TX, ntiles = ntz * ntx;
    const int c = blockIdx.x / ntiles, tile = blockIdx.x - c * ntiles;
    const int bz = tile / ntx, bx = tile - bz * ntx;
    const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
    const int iz0 = bz * 8, ixb = bx * TX;
    const int iz = iz0 + ty, ix0 = ixb + 4 * tx;
    const int s0 = c * chunk, s1 = min(ns, s0 + chunk), nsh = max(0, s1 - s0);
    // Pieces of rows below the model or of columns past nx + WL are not
    // copied: only points outside the model (never stored) read them. With
    // the sponge width a multiple of 4 the pieces start on 16-byte
    // boundaries (this thread's two: fixed offsets, precomputed); otherwise
    // they are copied 4 bytes at a time.
    const bool al = (L.P & 3) == 0;
    long long g0 = -1, g1 = -1;
    int d0 = 0, d1 = 0;
    {
        int r = threadIdx.x / (RW / 4), c4 = threadIdx.x - r * (RW / 4), col = ixb - WL + 4 * c4;
        if (iz0 + r < L.nz && col < L.nx + WL) {
            g0 = fidx(L, iz0 + r + L.P, col + L.P);
            d0 = r * RW + 4 * c4;
        }
        const int e1 = threadIdx.x + TPB;
        if (e1 < NCH) {
            r = e1 / (RW / 4);
            c4 = e1 - r * (RW / 4);
            col = ixb - WL + 4 * c4;
            if (iz0 + r < L.nz && col < L.nx + WL) {
                g1 = fidx(L, iz0 + r + L.P, col + L.P);
                d1 = r * RW + 4 * c4;
            }
        }
    }
    // shots SPS k .. SPS k + SPS - 1 of the chunk into stage b (one commit group)
    auto stage = [&](int k, int b) {
#pragma unroll
        for (int q = 0; q < SPS; ++q) {
            const int s = s0 + SPS * k + q;
            if (s >= s1) break;
            const float *src = u + (long long)s * L.fstride;
            if (al) {
                if (g0 >= 0) cp_async16(&sm[b][q][d0], src + g0);
                if (g1 >= 0) cp_async16(&sm[b][q][d1], src + g1);
            } else {
                for (int e = threadIdx.x; e < 8 * RW; e += TPB) {
                    const int r = e / RW, cc = e - r * RW, col = ixb - WL + cc;
                    if (iz0 + r < L.nz && col < L.nx + WL)
                        cp_async4(&sm[b][q][r * RW + cc], src + fidx(L, iz0 + r + L.P, col + L.P));
                }
            }
        }
        asm volatile("cp.async.commit_group;" ::: "memory");
    };
    float2 acc[NHC][2];
#pragma unroll
    for (int h = 0; h < NHC; ++h) acc[h][0] = acc[h][1] = make_float2(0.f, 0.f);
    auto window = [&](const float *row, float (&w)[4 * NW]) {
#pragma unroll
        for (int kk = 0; kk < NW; ++kk) {
            const float4 t = lds4(row + 4 * kk);
            w[4 * kk] = t.x; w[4 * kk + 1] = t.y; w[4 * kk + 2] = t.z; w[4 * kk + 3] = t.w;
        }
    };
    // u(x+h) u(x-h); even h: points (0, 1) and (2, 3) on lane pairs; odd h:
    // (1, 2) paired, 0 and 3 scalar (as in the fused step)
    auto products = [&](const float (&w)[4 * NW]) {
#pragma unroll
        for (int h = 0; h < NHC; ++h) {
            if ((h & 1) == 0) {
#pragma unroll
                for (int qq = 0; qq < 2; ++qq)
                    acc[h][qq] = fma2(f2(w[WL + 2 * qq + h], w[WL + 2 * qq + 1 + h]),
                                      f2(w[WL + 2 * qq - h], w[WL + 2 * qq + 1 - h]), acc[h][qq]);
            } else {
                acc[h][0] = fma2(f2(w[WL + 1 + h], w[WL + 2 + h]), f2(w[WL + 1 - h], w[WL + 2 - h]), acc[h][0]);
                acc[h][1].x = fmaf(w[WL + h], w[WL - h], acc[h][1].x);
                acc[h][1].y = fmaf(w[WL + 3 + h], w[WL + 3 - h], acc[h][1].y);
            }
        }
    };
    const int nstage = (nsh + SPS - 1) / SPS;
#pragma unroll
    for (int k = 0; k < NST - 1; ++k) {
        if (k < nstage) stage(k, k);
        else asm volatile("cp.async.commit_group;" ::: "memory");
    }
#pragma unroll 1
    for (int k = 0; k < nstage; ++k) {
        // the group of stage k is complete when at most NST - 2 younger ones are pending
        asm volatile("cp.async.wait_group %0;" ::"n"(NST - 2) : "memory");
        __syncthreads(); // stage k visible to all; stage k - 1's slot free for reuse
        if (k + NST - 1 < nstage) stage(k + NST - 1, (k + NST - 1) % NST);
        else asm volatile("cp.async.commit_group;" ::: "memory");
        const int nq = min(SPS, nsh - SPS * k);
        const int b = k % NST;
#pragma unroll 1
        for (int q = 0; q < nq; q += 2) {
            float w0[4 * NW];
            window(&sm[b][q][ty * RW + 4 * tx], w0);
            if (q + 1 < nq) { // shots in order: q, then q + 1
                float w1[4 * NW];
                window(&sm[b][q + 1][ty * RW + 4 * tx], w1);
                products(w0);
                products(w1);
            } else {
                products(w0);
            }
        }
    }
    asm volatile("cp.async.wait_all;" ::: "memory");
    if (iz >= L.nz || ix0 >= L.nx) return;
    const long long nphys = (long long)L.nz * L.nx, o = (long long)iz * L.nx + ix0;
    const bool vec = ((L.P | L.nx) & 3) == 0 && ix0 + 3 < L.nx;
#pragma unroll
    for (int h = 0; h < NHC; ++h) {
        if (h > hmax) continue;
        const float v[4] = {(h & 1) ? acc[h][1].x : acc[h][0].x, (h & 1) ? acc[h][0].x : acc[h][0].y,
                            (h & 1) ? acc[h][0].y : acc[h][1].x, acc[h][1].y};
        if (vec) {
            red_add4(acc_offh + h * nphys + o, v[0], v[1], v[2], v[3]);
        } else {
#pragma unroll
            for (int p = 0; p < 4; ++p)
                if (ix0 + p < L.nx) atomicAdd(acc_offh + h * nphys + o + p, v[p]);
        }
    }
}

// ---------------------------------------------------------------- launchers
namespace {
// Compiled tile variants of each kind of step (index 0 is the default; the
// autotuner may pick another per problem shape): tile height 8 RZ rows,
// ring stages, minimum resident CTAs per SM (the register cap).
struct Variant {
    int rz, spi, smem; // tile rows / 8, shots per item, dynamic shared memory
    int nh;            // offsets of the offset Hessian it accumulates (valid for hmax <= nh - 1)
    int split;         // offset Hessian: 1 = the plain step, then k_offh_level
    const void *fn[3]; // one model per launch, batch of up to BATCH_MAX models, and (plain
                       // forward and backward steps) the one-model instance that keeps (forward)
                       // or reads (backward) the imaging factor q of a re-propagated segment
    int occ[2];        // resident CTAs per SM (from the occupancy calculator)
};

#define FWD_VARIANT(RZ, ST, MINB, SPI)                                                     \
    {RZ, SPI, FwdRing<RZ, RADIUS, false, ST, SPI>::SMEM, 0, 0,                             \
     {(const void *)k_fwd_step<RZ, RADIUS, false, ST, MINB, 1, SPI>,                       \
      (const void *)k_fwd_step<RZ, RADIUS, false, ST, MINB, BATCH_MAX, SPI>,               \
      (const void *)k_fwd_step<RZ, RADIUS, false, ST, MINB, 1, SPI, HMAX_LIMIT + 1, true>}, \
     {0, 0}}
#define FWDH_VARIANT(ST, MINB, SPI, NHC)                                                   \
    {1, SPI, FwdRing<1, HMAX_LIMIT, true, ST, SPI>::SMEM, NHC, 0,                          \
     {(const void *)k_fwd_step<1, HMAX_LIMIT, true, ST, MINB, 1, SPI, NHC>,                \
      (const void *)k_fwd_step<1, HMAX_LIMIT, true, ST, MINB, BATCH_MAX, SPI, NHC>, nullptr}, \
     {0, 0}}
// the plain step with the offset Hessian summed by k_offh_level after it
#define FWDS_VARIANT(RZ, ST, MINB, SPI)                                                    \
    {RZ, SPI, FwdRing<RZ, RADIUS, false, ST, SPI>::SMEM, HMAX_LIMIT + 1, 1,               \
     {(const void *)k_fwd_step<RZ, RADIUS, false, ST, MINB, 1, SPI>,                       \
      (const void *)k_fwd_step<RZ, RADIUS, false, ST, MINB, BATCH_MAX, SPI>, nullptr},     \
     {0, 0}}
#define BWD_VARIANT(RZ, ST, MINB)                                                          \
    {RZ, 1, BwdRing<RZ, ST>::SMEM, 0, 0,                                                   \
     {(const void *)k_bwd_step<RZ, ST, MINB, 1>, (const void *)k_bwd_step<RZ, ST, MINB, BATCH_MAX>, \
      (const void *)k_bwd_step<RZ, ST, MINB, 1, 0, true>},                                \
     {0, 0}}

// forward: 64 x 16 tiles (3 stages, 4 CTAs/SM), 64 x 32 (2 stages), 64 x 8
// (6 CTAs/SM), 64 x 16 with two shots per item (2 stages)
Variant g_var_f[] = {FWD_VARIANT(2, 3, 4, 1), FWD_VARIANT(4, 2, 4, 1), FWD_VARIANT(1, 3, 6, 1),
                     FWD_VARIANT(2, 2, 4, 2)};
// forward with the offset Hessian: fused, 64 x 8 tiles, halo 12 (its 44
// register accumulators rule out taller tiles), one or two shots per item
// (the accumulators serve both shots of an item) and the offset count
// compiled for hmax <= 12 or <= 10; split, the plain step (64 x 16 tiles, one
// or two shots per item) and k_offh_level
Variant g_var_h[] = {FWDH_VARIANT(3, 4, 1, 13), FWDH_VARIANT(3, 4, 2, 13), FWDH_VARIANT(3, 4, 2, 11),
                     FWDS_VARIANT(2, 3, 4, 1), FWDS_VARIANT(2, 2, 4, 2)};
// backward: 64 x 16 tiles (2 stages, 4 CTAs/SM), 64 x 8 (5 CTAs/SM)
Variant g_var_b[] = {BWD_VARIANT(2, 2, 4), BWD_VARIANT(1, 2, 5)};

Variant *variants(StepKind k, int &n)
{
    if (k == STEP_FWD) {
        n = (int)(sizeof g_var_f / sizeof g_var_f[0]);
        return g_var_f;
    }
    if (k == STEP_FWD_OFFH) {
        n = (int)(sizeof g_var_h / sizeof g_var_h[0]);
        return g_var_h;
    }
    n = (int)(sizeof g_var_b / sizeof g_var_b[0]);
    return g_var_b;
}

// shots per chunk tried by the autotuner (index 0 = default of the kind)
const int CHUNKS_F[] = {8, 16};
const int CHUNKS_H[] = {16, 8};

std::once_flag g_prep_once;

void prepare_kernels()
{
    std::call_once(g_prep_once, [] {
        int dev = 0;
        const bool have_dev = cudaGetDevice(&dev) == cudaSuccess;
        for (int k = 0; k < 3; ++k) {
            int n = 0;
            Variant *v = variants((StepKind)k, n);
            for (int i = 0; i < n; ++i)
                for (int b = 0; b < 2; ++b) {
                    int occ = 0;
                    if (have_dev) {
                        cudaFuncSetAttribute(v[i].fn[b], cudaFuncAttributeMaxDynamicSharedMemorySize, v[i].smem);
                        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, v[i].fn[b], TPB, v[i].smem) !=
                            cudaSuccess)
                            occ = 0;
                    }
                    v[i].occ[b] = occ > 0 ? occ : 2;
                }
            for (int i = 0; i < n; ++i)
                if (have_dev && v[i].fn[2])
                    cudaFuncSetAttribute(v[i].fn[2], cudaFuncAttributeMaxDynamicSharedMemorySize, v[i].smem);
        }
        cudaGetLastError();
    });
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

// shot blocks of a model's level: blocks of `chunk` shots, the last one cut in
// two when there are two or more (cursor_set)
int chunk_blocks(int ns, int chunk)
{
    const int nb = (ns + chunk - 1) / chunk;
    return nb == 1 ? 1 : nb - 1 + (ns - (nb - 1) * chunk >= 2 ? 2 : 1);
}

// autotuned (variant, chunk) per problem shape
struct TuneKey {
    int kind, nzp, nxp, ns;
    bool operator<(const TuneKey &o) const
    {
        return std::tie(kind, nzp, nxp, ns) < std::tie(o.kind, o.nzp, o.nxp, o.ns);
    }
};
std::mutex g_tune_mu;
std::map<TuneKey, std::pair<int, int>> g_tuned;

// chunk counts of a launch's models and the number of CTAs to launch
template <class A, int N>
int batch_fill(Batch<A, N> &b, const A *a, const Tiling *t, int nm, int occ)
{
    long long total = 0;
    for (int k = 0; k < nm; ++k) {
        b.m[k] = a[k];
        total += (long long)t[k].ntx * t[k].ntz * chunk_blocks(a[k].c.ns, t[0].chunk);
        b.chunk_end[k] = (int)total;
    }
    for (int k = nm; k < N; ++k) b.chunk_end[k] = (int)total;
    b.nm = nm;
    b.chunk = t[0].chunk;
    b.sched = a[0].c.sched;
    const long long slots = (long long)sm_count_dev() * occ;
    return (int)(total < slots ? total : slots);
}

template <class A, int N>
cudaError_t launch_variant(const Variant &v, int b, Batch<A, N> &args, int ctas, cudaStream_t st)
{
    if (ctas <= 0) return cudaSuccess;
    void *params[] = {&args};
    return cudaLaunchKernel(v.fn[b], dim3(ctas), dim3(TPB), params, (size_t)v.smem, st);
}
} // namespace

int step_variants(StepKind kind)
{
    int n = 0;
    variants(kind, n);
    return n;
}

int step_chunks(StepKind kind, const int **chunks)
{
    *chunks = kind == STEP_FWD_OFFH ? CHUNKS_H : CHUNKS_F;
    return 2;
}

void step_tuned_store(StepKind kind, const Lay2D &L, int ns, int variant, int chunk)
{
    std::lock_guard<std::mutex> lock(g_tune_mu);
    g_tuned[TuneKey{kind, L.nzp, L.nxp, ns}] = {variant, chunk};
}

bool step_tuned_lookup(StepKind kind, const Lay2D &L, int ns, int &variant, int &chunk)
{
    std::lock_guard<std::mutex> lock(g_tune_mu);
    auto it = g_tuned.find(TuneKey{kind, L.nzp, L.nxp, ns});
    if (it == g_tuned.end()) return false;
    variant = it->second.first;
    chunk = it->second.second;
    return true;
}

void step_tuned_clear()
{
    std::lock_guard<std::mutex> lock(g_tune_mu);
    g_tuned.clear();
}

void step_boxes(StepKind kind, const Tiling &t, int &hx, int &hy, int &px, int &py)
{
    int n = 0;
    const bool fused_h = kind == STEP_FWD_OFFH && !variants(kind, n)[t.variant].split;
    const int halo = fused_h ? HMAX_LIMIT : RADIUS;
    hx = TX + 2 * halo;
    hy = t.tz + 2 * RADIUS;
    px = TX;
    py = t.tz;
}

int max_tiles(const Lay2D &L) { return ((L.nxp + TX - 1) / TX) * ((L.nzp + 7) / 8); }

bool step_variant_valid(StepKind kind, int variant, int hmax)
{
    int n = 0;
    Variant *vs = variants(kind, n);
    if (variant < 0 || variant >= n) return false;
    return kind != STEP_FWD_OFFH || hmax <= vs[variant].nh - 1;
}

Tiling make_tiling(const Lay2D &L, int ns, StepKind kind, int variant, int chunk, int hmax)
{
    prepare_kernels();
    int n = 0;
    Variant *vs = variants(kind, n);
    if (!step_variant_valid(kind, variant, hmax)) {
        int tv = 0, tc = 0;
        if (step_tuned_lookup(kind, L, ns, tv, tc) && step_variant_valid(kind, tv, hmax)) {
            variant = tv;
            if (chunk <= 0) chunk = tc;
        } else {
            // default: the first variant, or for the offset Hessian the one
            // with the fewest offsets that covers hmax, two shots per item
            variant = 0;
            if (kind == STEP_FWD_OFFH)
                for (int i = 0; i < n; ++i)
                    if (vs[i].spi == 2 && hmax <= vs[i].nh - 1 &&
                        (!step_variant_valid(kind, variant, hmax) || vs[variant].spi != 2 || vs[i].nh < vs[variant].nh))
                        variant = i;
        }
    }
    if (chunk <= 0) chunk = kind == STEP_FWD_OFFH ? CHUNKS_H[0] : CHUNKS_F[0];
    Tiling t;
    t.variant = variant;
    t.spi = vs[variant].spi;
    t.tz = 8 * vs[variant].rz;
    t.ntx = (L.nxp + TX - 1) / TX;
    t.ntz = (L.nzp + t.tz - 1) / t.tz;
    const int tiles = t.ntx * t.ntz;
    t.chunk = chunk > ns ? ns : chunk;
    const long long chunks = (long long)tiles * chunk_blocks(ns, t.chunk);
    const long long slots = (long long)sm_count_dev() * vs[variant].occ[0];
    t.ctas = (int)(chunks < slots ? chunks : slots);
    return t;
}

namespace {
// k_offh_level for one model's level (split variants): a chunk of shots per
// tile such that the tiles x chunks fill the resident CTAs about once
cudaError_t launch_offh_sums(const FwdArgs &a, cudaStream_t st)
{
    if (a.acc_offh == nullptr || a.uin == nullptr) return a.acc_offh == nullptr ? cudaSuccess : cudaErrorInvalidValue;
    static int occ = 0;
    if (occ == 0) {
        int o = 0;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&o, k_offh_level<13, 3, 4>, TPB, 0) != cudaSuccess || o <= 0) o = 4;
        cudaGetLastError();
        occ = o;
    }
    const Lay2D &L = a.c.L;
    const int ns = a.c.ns;
    const int ntiles = ((L.nz + 7) / 8) * ((L.nx + TX - 1) / TX);
    const int nch = std::max(1, std::min(ns, sm_count_dev() * occ / std::max(1, ntiles)));
    const int chunk = ((ns + nch - 1) / nch + 1) & ~1;
    const int grid = ntiles * ((ns + chunk - 1) / chunk);
    if (a.hmax <= 10)
        k_offh_level<11, 3, 4><<<grid, TPB, 0, st>>>(a.uin, L, ns, chunk, a.hmax, a.acc_offh);
    else
        k_offh_level<13, 3, 4><<<grid, TPB, 0, st>>>(a.uin, L, ns, chunk, a.hmax, a.acc_offh);
    return cudaGetLastError();
}
} // namespace

bool fwd_split(const Tiling &t, bool with_offh)
{
    int n = 0;
    return with_offh && variants(STEP_FWD_OFFH, n)[t.variant].split != 0;
}

cudaError_t launch_fwd_step(const FwdArgs &a, const Tiling &t, bool with_offh, cudaStream_t st)
{
    int n = 0;
    const Variant &v = variants(with_offh ? STEP_FWD_OFFH : STEP_FWD, n)[t.variant];
    if (a.qout != nullptr && (with_offh || !v.fn[2])) return cudaErrorInvalidValue;
    if (a.qout == nullptr && a.uout == nullptr) return cudaErrorInvalidValue;
    Batch<FwdArgs, 1> b;
    cudaError_t e = launch_variant(v, a.qout != nullptr ? 2 : 0, b, batch_fill(b, &a, &t, 1, v.occ[0]), st);
    if (e == cudaSuccess && with_offh && v.split) e = launch_offh_sums(a, st);
    return e;
}

cudaError_t launch_bwd_step(const BwdArgs &a, const Tiling &t, cudaStream_t st)
{
    int n = 0;
    const Variant &v = variants(STEP_BWD, n)[t.variant];
    if (a.qin && (a.recon || !v.fn[2])) return cudaErrorInvalidValue;
    Batch<BwdArgs, 1> b;
    return launch_variant(v, a.qin ? 2 : 0, b, batch_fill(b, &a, &t, 1, v.occ[0]), st);
}

cudaError_t launch_fwd_batch(const FwdArgs *a, const Tiling *t, int nm, bool with_offh, cudaStream_t st)
{
    if (nm < 1 || nm > BATCH_MAX) return cudaErrorInvalidValue;
    int n = 0;
    const Variant &v = variants(with_offh ? STEP_FWD_OFFH : STEP_FWD, n)[t[0].variant];
    Batch<FwdArgs, BATCH_MAX> b;
    cudaError_t e = launch_variant(v, 1, b, batch_fill(b, a, t, nm, v.occ[1]), st);
    for (int k = 0; k < nm && e == cudaSuccess && with_offh && v.split; ++k) e = launch_offh_sums(a[k], st);
    return e;
}

cudaError_t launch_bwd_batch(const BwdArgs *a, const Tiling *t, int nm, cudaStream_t st)
{
    if (nm < 1 || nm > BATCH_MAX) return cudaErrorInvalidValue;
    int n = 0;
    const Variant &v = variants(STEP_BWD, n)[t[0].variant];
    Batch<BwdArgs, BATCH_MAX> b;
    return launch_variant(v, 1, b, batch_fill(b, a, t, nm, v.occ[1]), st);
}

namespace {
constexpr int BORN_RZ = 2, BORN_ST = 2, BORN_MINB = 4;
#define K_BORN k_born_step<BORN_RZ, BORN_ST, BORN_MINB>
constexpr int SMEM_BORN = BornRing<BORN_RZ, BORN_ST>::SMEM;
std::once_flag g_born_once;
int g_occ_born = 2;
} // namespace

// ---------------------------------------------------- extended operators
namespace {
template <int HE> struct ExtKernels {
    static constexpr int SMEM_B = BwdRingE<1, 2, HE>::SMEM;
    static constexpr int SMEM_O = BornRingE<1, 2, HE>::SMEM;
    static std::once_flag once;
    static int occ_b, occ_o;
    static void prepare()
    {
        std::call_once(once, [] {
            auto kb = k_bwd_step<1, 2, 3, 1, HE>;
            auto ko = k_born_step<1, 2, 3, HE>;
            cudaFuncSetAttribute(kb, cudaFuncAttributeMaxDynamicSharedMemorySize, SMEM_B);
            cudaFuncSetAttribute(ko, cudaFuncAttributeMaxDynamicSharedMemorySize, SMEM_O);
            int o = 0;
            if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&o, kb, TPB, SMEM_B) == cudaSuccess && o > 0) occ_b = o;
            if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&o, ko, TPB, SMEM_O) == cudaSuccess && o > 0) occ_o = o;
            cudaGetLastError();
        });
    }
    static cudaError_t bwd(const BwdArgs &a, const Tiling &t, cudaStream_t st)
    {
        prepare();
        Batch<BwdArgs, 1> b;
        const int ctas = batch_fill(b, &a, &t, 1, occ_b);
        if (ctas <= 0) return cudaSuccess;
        k_bwd_step<1, 2, 3, 1, HE><<<ctas, TPB, SMEM_B, st>>>(b);
        return cudaGetLastError();
    }
    static cudaError_t born(const BornArgs &a, const Tiling &t, cudaStream_t st)
    {
        prepare();
        Batch<BornArgs, 1> b;
        const int ctas = batch_fill(b, &a, &t, 1, occ_o);
        if (ctas <= 0) return cudaSuccess;
        k_born_step<1, 2, 3, HE><<<ctas, TPB, SMEM_O, st>>>(b);
        return cudaGetLastError();
    }
};
template <int HE> std::once_flag ExtKernels<HE>::once;
template <int HE> int ExtKernels<HE>::occ_b = 1;
template <int HE> int ExtKernels<HE>::occ_o = 1;
} // namespace

int ext_kernel_he(int hext) { return hext <= 2 ? 2 : (hext <= 4 ? 4 : 6); }

void ext_boxes(int he, const Tiling &t, int &hx, int &hy, int &px, int &py)
{
    hx = TX + 2 * (RADIUS + 2 * he);
    hy = t.tz + 2 * RADIUS;
    px = TX;
    py = t.tz;
}

cudaError_t launch_bwd_ext_step(const BwdArgs &a, const Tiling &t, int he, cudaStream_t st)
{
    if (t.tz != 8) return cudaErrorInvalidValue;
    switch (he) {
    case 2: return ExtKernels<2>::bwd(a, t, st);
    case 4: return ExtKernels<4>::bwd(a, t, st);
    case 6: return ExtKernels<6>::bwd(a, t, st);
    default: return cudaErrorInvalidValue;
    }
}

cudaError_t launch_born_ext_step(const BornArgs &a, const Tiling &t, int he, cudaStream_t st)
{
    if (t.tz != 8) return cudaErrorInvalidValue;
    switch (he) {
    case 2: return ExtKernels<2>::born(a, t, st);
    case 4: return ExtKernels<4>::born(a, t, st);
    case 6: return ExtKernels<6>::born(a, t, st);
    default: return cudaErrorInvalidValue;
    }
}

cudaError_t launch_born_step(const BornArgs &a, const Tiling &t, cudaStream_t st)
{
    std::call_once(g_born_once, [] {
        cudaFuncSetAttribute(K_BORN, cudaFuncAttributeMaxDynamicSharedMemorySize, SMEM_BORN);
        int occ = 0;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, K_BORN, TPB, SMEM_BORN) == cudaSuccess && occ > 0)
            g_occ_born = occ;
        cudaGetLastError();
    });
    if (t.tz != 8 * BORN_RZ) return cudaErrorInvalidValue;
    Batch<BornArgs, 1> b;
    const int ctas = batch_fill(b, &a, &t, 1, g_occ_born);
    if (ctas <= 0) return cudaSuccess;
    K_BORN<<<ctas, TPB, SMEM_BORN, st>>>(b);
    return cudaGetLastError();
}

// Tensor map over `nfields` stored fields [nfields][rows][pitch] (float32)
// with a box of bx x by cells; out-of-range cells read as zero.
bool encode_field_map(CUtensorMap *map, const float *base, const Lay2D &L, int nfields, int bx, int by, int bz)
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
    const cuuint32_t box[3] = {(cuuint32_t)bx, (cuuint32_t)by, (cuuint32_t)bz};
    const cuuint32_t estr[3] = {1, 1, 1};
    CUresult r = encode(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, const_cast<float *>(base), dims, strides, box,
                        estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                        CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS;
}

} // namespace fwi
