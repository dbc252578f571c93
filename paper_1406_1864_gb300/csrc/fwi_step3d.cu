// fwi_step3d.cu -- time-step kernels of the 3-D FWI gradient (sm_103a).
//
// The same discrete scheme as in 2-D [Sec. 2]: damped leapfrog with the
// 8th-order Laplacian, now over three axes (25 points),
//   u^{n+1} = u^n + fma(c2 ia, Lhat u^n + f delta_s / dx, (2 ia - 1)(u^n - u^{n-1})),
// ia = 1/(1 + eta dt) per cell (1 in the model, where the update is exactly
// the plain leapfrog), traces d^n = R u^n, the illumination of Eq. 1, and
// in the backward step the adjoint psi^m of the same update with the
// residuals injected at the receivers (dx^2 R^T a^m) and the zero-lag
// imaging sum psi^m (Lhat u^{m-1} + f delta_s / dx).
//
// Work decomposition (GB300-first): a CTA of 128 threads owns one column of
// 64 (x) x 8 (y) cells of one shot and marches it down z. Each thread keeps
// its 4 x-points' values of the nine planes i-4 .. i+4 in registers (the z
// part of the stencil); for the x and y parts, plane i with its 4-cell halo is
// brought into shared memory by a 4-D TMA copy (x, y, z, shot), together with
// the point tile of plane i+4 that enters the register window and the point
// tiles of u^{n-1}, c2 and the damping factor of plane i: one ring stage per
// plane, STAGES-1 planes ahead of the compute, on mbarriers with bounded
// waits. A column may be cut into z-segments, so that the items (segment,
// column, shot) come in units fine enough for the last round of a launch to
// keep the SMs busy; a segment's march starts with its window planes loaded
// straight from global memory. Items are handed out by an atomic counter,
// segment-major, the shots of one column consecutively, so neighbouring
// columns are in flight together and their halo re-reads hit L2.
// Accumulations (illumination, gradient) are red.add per point and plane: a
// column's planes do not fit in registers.
#include "fwi_device.cuh"

#include <algorithm>
#include <map>
#include <mutex>
#include <tuple>

namespace fwi {
namespace {

constexpr int TXS3 = TX + 2 * RADIUS;             // halo row length
constexpr int HALO3 = (TY3 + 2 * RADIUS) * TXS3;  // floats of one halo plane tile
constexpr int PT3 = TY3 * TX;                     // floats of one point tile

struct Item3 {
    int tile, s; // tile < 0: no more work
    int z0, z1;  // planes z0 .. z1 - 1 of the column
};

__device__ __forceinline__ void tma_load_4d(uint32_t dst, const CUtensorMap *map, int x, int y, int z, int w,
                                            uint32_t bar)
{
    asm volatile("cp.async.bulk.tensor.4d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
                 " [%0], [%1, {%2, %3, %4, %5}], [%6];" ::"r"(dst),
                 "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(z), "r"(w), "r"(bar)
                 : "memory");
}

// Lhat in second-difference form over three axes for two adjacent points:
// sum_k W_k ((x_{-k}+x_{+k}-2c) + (y_{-k}+y_{+k}-2c) + (z_{-k}+z_{+k}-2c))
__device__ __forceinline__ float2 lap3x2(float2 c, const float2 (&xs)[4], const float2 (&ys)[4],
                                         const float2 (&zs)[4])
{
    const float2 m2 = make_float2(-2.f, -2.f);
    float2 q = mul2(make_float2(W4, W4),
                    add2(add2(fma2(c, m2, xs[3]), fma2(c, m2, ys[3])), fma2(c, m2, zs[3])));
    q = fma2(make_float2(W3, W3), add2(add2(fma2(c, m2, xs[2]), fma2(c, m2, ys[2])), fma2(c, m2, zs[2])), q);
    q = fma2(make_float2(W2, W2), add2(add2(fma2(c, m2, xs[1]), fma2(c, m2, ys[1])), fma2(c, m2, zs[1])), q);
    q = fma2(make_float2(W1, W1), add2(add2(fma2(c, m2, xs[0]), fma2(c, m2, ys[0])), fma2(c, m2, zs[0])), q);
    return q;
}

// Lhat of the thread's 4 points at the plane whose halo tile is `sh` (the
// thread's row at ty + RADIUS) with the z window zw (zw[4] = this plane)
__device__ __forceinline__ void lap3_4(float2 (&q)[2], const float *sh, const float4 (&zw)[9], int tx, int ty)
{
    const float *row = &sh[(ty + RADIUS) * TXS3 + RADIUS + 4 * tx];
    const float4 a0 = lds4(row - 4), a1 = lds4(row), a2 = lds4(row + 4);
    const float w[12] = {a0.x, a0.y, a0.z, a0.w, a1.x, a1.y, a1.z, a1.w, a2.x, a2.y, a2.z, a2.w};
    float4 yv[8];
#pragma unroll
    for (int k = 1; k <= RADIUS; ++k) {
        yv[k - 1] = lds4(row - k * TXS3);
        yv[k + 3] = lds4(row + k * TXS3);
    }
#pragma unroll
    for (int h = 0; h < 2; ++h) {
        const int p = 4 + 2 * h;
        float2 xs[4], ys[4], zs[4];
#pragma unroll
        for (int k = 1; k <= 4; ++k) {
            xs[k - 1] = f2(w[p - k] + w[p + k], w[p + 1 - k] + w[p + 1 + k]);
            ys[k - 1] = add2(half2of(yv[k - 1], h), half2of(yv[k + 3], h));
            zs[k - 1] = add2(half2of(zw[4 - k], h), half2of(zw[4 + k], h));
        }
        q[h] = lap3x2(f2(w[p], w[p + 1]), xs, ys, zs);
    }
}

// next item of this CTA (thread 0): segment-major, then columns in order,
// the shots of one column consecutively (CTAs running at the same time add
// into the same column of the imaging and illumination sums, which then stay
// in L2)
__device__ __forceinline__ Item3 grab_item(const Step3Common &c, int ntiles)
{
    const int q = atomicAdd(c.sched, 1);
    const int per = ntiles * c.ns; // items of one segment
    if (q >= per * c.nseg) return Item3{-1, 0, 0, 0};
    const int g = q / per, r = q - g * per;
    const int tile = r / c.ns;
    const int z0 = g * c.segl;
    return Item3{tile, r - tile * c.ns, z0, min(c.L.nzp, z0 + c.segl)};
}

// the thread's 4 points of planes z0 - 4 .. z0 + 3 of field f (rows k0 >= nyp
// or columns j0 >= nxp: zeros), the z window at the start of a segment;
// planes above the grid are the zero ghost planes
__device__ __forceinline__ void load_window(float4 (&zw)[9], const float *f, const Lay3D &L, int z0, int k0, int j0)
{
    const bool ok = k0 < L.nyp && j0 < L.nxp; // j0 + 3 stays inside the row's ghost columns
    const float *b = f + fidx3(L, z0 - 4, k0, j0);
#pragma unroll
    for (int z = 0; z < 8; ++z)
        zw[z] = (ok && z0 - 4 + z >= 0) ? __ldg(reinterpret_cast<const float4 *>(b + z * L.plane))
                                        : make_float4(0.f, 0.f, 0.f, 0.f);
    zw[8] = make_float4(0.f, 0.f, 0.f, 0.f);
}

// ------------------------------------------------------------ forward step
// stage: [halo u(i)] [u(i+4)] [u_prev(i)] [c2(i)] [damp(i)]
constexpr int FWD3_STAGE_F = HALO3 + 4 * PT3;

// QOUT: also store q^n (a.qout) and skip u^{n+1} where a.uout is null (the
// segments' re-propagation); otherwise neither test is compiled
template <int STAGES, int MINB, bool QOUT = false>
__global__ void __launch_bounds__(TPB, MINB) k_fwd3d(const __grid_constant__ Fwd3Args a)
{
    constexpr int D = STAGES - 1;
    static_assert(D >= 1, "at least two stages");
    extern __shared__ unsigned char smem_raw[];
    __shared__ int s_abort;
    __shared__ Item3 s_item[4];
    unsigned char *smem = align_smem(smem_raw);
    uint64_t *bars = reinterpret_cast<uint64_t *>(smem);
    float *ring = reinterpret_cast<float *>(smem + 128);

    const Step3Common &c = a.c;
    const Lay3D &L = c.L;
    const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
    const int ntiles = c.nty * c.ntx;

    if (threadIdx.x == 0) {
        for (int k = 0; k < STAGES; ++k) mbar_init(smem_u32(&bars[k]), 1);
        fence_mbar_init();
        s_abort = 0;
    }
    __syncthreads();

    // thread 0: copies of global step t = 0, 1, 2, ..., one plane of an item
    // per step: the item and plane are counted, the tile origin taken once per
    // item (no division per plane on the issuing warp)
    Item3 iss{-1, 0, 0, 0};
    int i_slot = 0, i_ls = 0, i_n = 1, ibk = 0, ibj = 0;
    auto issue = [&](int t) {
        if (i_ls == 0) {
            iss = grab_item(c, ntiles);
            s_item[i_slot & 3] = iss;
            if (iss.tile >= 0) {
                const int tz = iss.tile / c.ntx;
                ibk = tz * TY3;
                ibj = (iss.tile - tz * c.ntx) * TX;
                i_n = iss.z1 - iss.z0;
            }
        }
        if (iss.tile < 0) return; // no more items
        const int i = iss.z0 + i_ls;
        if (++i_ls == i_n) {
            i_ls = 0;
            ++i_slot;
        }
        const int bk = ibk, bj = ibj;
        const int st = t % STAGES;
        float *sg = ring + st * FWD3_STAGE_F;
        const uint32_t bar = smem_u32(&bars[st]);
        fence_proxy_async_smem();
        mbar_expect_tx(bar, (HALO3 + 4 * PT3) * 4);
        tma_load_4d(smem_u32(sg + HALO3), &a.tm_upt, GXL + bj, bk + GY, i + RADIUS + GZ, iss.s, bar);
        tma_load_4d(smem_u32(sg), &a.tm_u, GXL + bj - RADIUS, bk + GY - RADIUS, i + GZ, iss.s, bar);
        tma_load_4d(smem_u32(sg + HALO3 + PT3), &a.tm_prev, GXL + bj, bk + GY, i + GZ, iss.s, bar);
        tma_load_4d(smem_u32(sg + HALO3 + 2 * PT3), &a.tm_c2, GXL + bj, bk + GY, i + GZ, 0, bar);
        tma_load_4d(smem_u32(sg + HALO3 + 3 * PT3), &a.tm_damp, GXL + bj, bk + GY, i + GZ, 0, bar);
    };
    if (threadIdx.x == 0)
        for (int t = 0; t < D; ++t) issue(t);
    __syncthreads();

    float4 zw[9];
    int slot = 0, ls = 0;
    Item3 it{-1, 0, 0, 0};
    int k0 = 0, j0 = 0, my_e = 0, re = 0, my_plane = 0x7fffffff;
    int4 src = make_int4(-1, -1, -1, 0);
    float amp = 0.f;
    bool rowok = false;
    for (int t = 0;; ++t) {
        if (threadIdx.x == 0) issue(t + D);
        if (ls == 0) {
            it = s_item[slot & 3];
            if (it.tile < 0) break;
            const int bk = (it.tile / c.ntx) * TY3, bj = (it.tile % c.ntx) * TX;
            k0 = bk + ty;
            j0 = bj + 4 * tx;
            rowok = k0 < L.nyp;
            load_window(zw, a.uin + (long long)it.s * L.fstride, L, it.z0, k0, j0);
            src = c.src[it.s];
            amp = a.last ? 0.f : c.wav[(long long)it.s * c.nt + a.n] * c.src_scale;
            re = 0;
            my_plane = 0x7fffffff;
            if (a.seis != nullptr) {
                const int e0 = a.rt.ptr[it.tile * c.ns + it.s];
                re = a.rt.ptr[it.tile * c.ns + it.s + 1];
                my_e = e0 + (int)threadIdx.x;
                if (my_e < re) my_plane = a.rt.ent[my_e].x;
                while (my_plane < it.z0) { // entries of the segments above
                    my_e += TPB;
                    my_plane = my_e < re ? a.rt.ent[my_e].x : 0x7fffffff;
                }
            }
        }
        const int st = t % STAGES;
        const bool ok = stage_ready<STAGES>(bars, t, &s_abort);
        if (ok) {
            const float *sg = ring + st * FWD3_STAGE_F;
            zw[8] = lds4(&sg[HALO3 + ty * TX + 4 * tx]);
            const int i = it.z0 + ls;
            {
                const float4 cu = zw[4];
                const float2 u0[2] = {lo2(cu), hi2(cu)};
                float2 out[2] = {u0[0], u0[1]};
                const long long so = (long long)it.s * L.fstride;
                if (!a.last) {
                    float2 q[2];
                    lap3_4(q, sg, zw, tx, ty);
                    if (i == src.x && k0 == src.y) {
                        const int d = src.z - j0;
                        if (d == 0) q[0].x += amp;
                        if (d == 1) q[0].y += amp;
                        if (d == 2) q[1].x += amp;
                        if (d == 3) q[1].y += amp;
                    }
                    const float4 um4 = lds4(&sg[HALO3 + PT3 + ty * TX + 4 * tx]);
                    const float4 c24 = lds4(&sg[HALO3 + 2 * PT3 + ty * TX + 4 * tx]);
                    const float4 ia4 = lds4(&sg[HALO3 + 3 * PT3 + ty * TX + 4 * tx]);
#pragma unroll
                    for (int h = 0; h < 2; ++h) {
                        const float2 ia2 = half2of(ia4, h);
                        const float2 kb = fma2(ia2, make_float2(2.f, 2.f), make_float2(-1.f, -1.f));
                        out[h] = add2(u0[h], fma2(mul2(half2of(c24, h), ia2), q[h],
                                                  mul2(kb, sub2(u0[h], half2of(um4, h)))));
                    }
                    if (rowok && j0 < L.nxp) {
                        if (!QOUT || a.uout != nullptr) {
                            const float o[4] = {out[0].x, out[0].y, out[1].x, out[1].y};
                            store4(a.uout + so + fidx3(L, i, k0, j0), j0, L.nxp, o);
                        }
                        if (QOUT) { // for the backward step's imaging
                            const float qv[4] = {q[0].x, q[0].y, q[1].x, q[1].y};
                            store4(a.qout + so + fidx3(L, i, k0, j0), j0, L.nxp, qv);
                        }
                    }
                    if (a.illum_utt && a.acc_illum != nullptr) {
                        // (u^{n+1} - 2u^n + u^{n-1})^2 replaces u^2
#pragma unroll
                        for (int h = 0; h < 2; ++h)
                            out[h] = add2(fma2(u0[h], make_float2(-2.f, -2.f), out[h]), half2of(um4, h));
                    }
                }
                // receiver extraction d^n = R u^n at this plane
                while (my_plane == i) {
                    const int4 en = a.rt.ent[my_e];
                    const int ly = en.y >> 6, lx = en.y & 63;
                    a.seis[((long long)it.s * c.nt + a.n) * c.nrec + en.z] =
                        sg[(ly + RADIUS) * TXS3 + RADIUS + lx];
                    my_e += TPB;
                    my_plane = my_e < re ? a.rt.ent[my_e].x : 0x7fffffff;
                }
                // illumination of Eq. 1 (physical cells)
                if (a.acc_illum != nullptr && rowok && i >= L.P && i < L.P + L.nz && k0 >= L.P &&
                    k0 < L.P + L.ny) {
                    const bool utt = a.illum_utt && !a.last;
                    const float2 e0 = utt ? out[0] : u0[0], e1 = utt ? out[1] : u0[1];
                    const float ev[4] = {e0.x, e0.y, e1.x, e1.y};
                    const long long rowb = ((long long)(i - L.P) * L.ny + (k0 - L.P)) * L.nx;
                    const int ix0 = j0 - L.P;
                    if (((L.P | L.nx) & 3) == 0 && ix0 >= 0 && ix0 + 3 < L.nx) {
                        red_add4(a.acc_illum + rowb + ix0, ev[0] * ev[0], ev[1] * ev[1], ev[2] * ev[2], ev[3] * ev[3]);
                    } else {
#pragma unroll
                        for (int p = 0; p < 4; ++p) {
                            const int ix = ix0 + p;
                            if (ix >= 0 && ix < L.nx) atomicAdd(a.acc_illum + rowb + ix, ev[p] * ev[p]);
                        }
                    }
                }
            }
        }
#pragma unroll
        for (int z = 0; z < 8; ++z) zw[z] = zw[z + 1];
        __syncthreads();
        if (s_abort) {
            if (threadIdx.x == 0) {
                atomicOr(c.status, ST_TIMEOUT);
                for (int j = t; j < t + STAGES; ++j) mbar_wait(smem_u32(&bars[j % STAGES]), (j / STAGES) & 1, 200000000ull);
            }
            return;
        }
        if (++ls == it.z1 - it.z0) {
            ls = 0;
            ++slot;
        }
    }
}

// ----------------------------------------------------------- backward step
// The imaging factor q^{m-1} = Lhat u^{m-1} + f delta_s / dx is the one the
// re-propagation's forward step m-1 computed (and kept): read as a point
// tile, bitwise the value a Laplacian here would give.
// stage: [halo psi(i)] [psi(i+4)] [psi_b(i)] [c2(i)] [damp(i)] [q(i)]
constexpr int BWD3_STAGE_F = HALO3 + 5 * PT3;

template <int STAGES, int MINB>
__global__ void __launch_bounds__(TPB, MINB) k_bwd3d(const __grid_constant__ Bwd3Args a)
{
    constexpr int D = STAGES - 1;
    static_assert(D >= 1, "at least two stages");
    extern __shared__ unsigned char smem_raw[];
    __shared__ int s_abort;
    __shared__ Item3 s_item[4];
    __shared__ __align__(16) float sinj[PT3]; // adjoint source of the current plane (read as float4)
    unsigned char *smem = align_smem(smem_raw);
    uint64_t *bars = reinterpret_cast<uint64_t *>(smem);
    float *ring = reinterpret_cast<float *>(smem + 128);

    const Step3Common &c = a.c;
    const Lay3D &L = c.L;
    const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
    const int ntiles = c.nty * c.ntx;
    const int m = a.m;

    if (threadIdx.x == 0) {
        for (int k = 0; k < STAGES; ++k) mbar_init(smem_u32(&bars[k]), 1);
        fence_mbar_init();
        s_abort = 0;
    }
    for (int e = threadIdx.x; e < PT3; e += TPB) sinj[e] = 0.f;
    __syncthreads();

    // (issue: as in the forward step, steps t = 0, 1, 2, ... counted)
    Item3 iss{-1, 0, 0, 0};
    // (plane i_z of the item of slot i_slot; the plane as the counter keeps
    // the step state to two registers)
    int i_slot = 0, i_z = 0, i_zend = 0, ibk = 0, ibj = 0;
    auto issue = [&](int t) {
        if (i_z == i_zend) {
            iss = grab_item(c, ntiles);
            s_item[i_slot & 3] = iss;
            if (iss.tile >= 0) {
                const int tz = iss.tile / c.ntx;
                ibk = tz * TY3;
                ibj = (iss.tile - tz * c.ntx) * TX;
                i_z = iss.z0;
                i_zend = iss.z1;
            }
        }
        if (iss.tile < 0) return; // no more items
        const int i = i_z;
        if (++i_z == i_zend) ++i_slot;
        const int bk = ibk, bj = ibj;
        const int st = t % STAGES;
        float *sg = ring + st * BWD3_STAGE_F;
        const uint32_t bar = smem_u32(&bars[st]);
        fence_proxy_async_smem();
        mbar_expect_tx(bar, (HALO3 + 5 * PT3) * 4);
        tma_load_4d(smem_u32(sg + HALO3), &a.tm_ppt, GXL + bj, bk + GY, i + RADIUS + GZ, iss.s, bar);
        tma_load_4d(smem_u32(sg), &a.tm_p, GXL + bj - RADIUS, bk + GY - RADIUS, i + GZ, iss.s, bar);
        tma_load_4d(smem_u32(sg + HALO3 + PT3), &a.tm_pb, GXL + bj, bk + GY, i + GZ, iss.s, bar);
        tma_load_4d(smem_u32(sg + HALO3 + 2 * PT3), &a.tm_c2, GXL + bj, bk + GY, i + GZ, 0, bar);
        tma_load_4d(smem_u32(sg + HALO3 + 3 * PT3), &a.tm_damp, GXL + bj, bk + GY, i + GZ, 0, bar);
        tma_load_4d(smem_u32(sg + HALO3 + 4 * PT3), &a.tm_q, GXL + bj, bk + GY, i + GZ, iss.s, bar);
    };
    if (threadIdx.x == 0)
        for (int t = 0; t < D; ++t) issue(t);
    __syncthreads();

    float4 zp[9];
    int slot = 0, zi = 0, zend = 0; // plane zi of the item of slot `slot`
    Item3 it{-1, 0, 0, 0};
    int k0 = 0, j0 = 0, my_e = 0, re = 0, my_plane = 0x7fffffff;
    int2 zr = make_int2(1, 0);
    bool rowok = false;
    for (int t = 0;; ++t) {
        if (threadIdx.x == 0) issue(t + D);
        if (zi == zend) {
            it = s_item[slot & 3];
            if (it.tile < 0) break;
            zi = it.z0;
            zend = it.z1;
            const int bk = (it.tile / c.ntx) * TY3, bj = (it.tile % c.ntx) * TX;
            k0 = bk + ty;
            j0 = bj + 4 * tx;
            rowok = k0 < L.nyp;
            load_window(zp, a.pin + (long long)it.s * L.fstride, L, it.z0, k0, j0);
            re = 0;
            my_plane = 0x7fffffff;
            zr = make_int2(1, 0);
            if (a.adj != nullptr) {
                const int e0 = a.rt.ptr[it.tile * c.ns + it.s];
                re = a.rt.ptr[it.tile * c.ns + it.s + 1];
                zr = a.rt.zr[it.tile * c.ns + it.s];
                my_e = e0 + (int)threadIdx.x;
                if (my_e < re) my_plane = a.rt.ent[my_e].x;
                while (my_plane < it.z0) { // entries of the segments above
                    my_e += TPB;
                    my_plane = my_e < re ? a.rt.ent[my_e].x : 0x7fffffff;
                }
            }
        }
        const int st = t % STAGES;
        const int i = zi;
        // adjoint source of this plane into shared memory (uniform test)
        const bool inj = i >= zr.x && i <= zr.y;
        if (inj) {
            while (my_plane == i) {
                const int4 en = a.rt.ent[my_e];
                atomicAdd(&sinj[en.y], a.adj[((long long)it.s * c.nt + m) * c.nrec + en.z] * a.adj_scale);
                my_e += TPB;
                my_plane = my_e < re ? a.rt.ent[my_e].x : 0x7fffffff;
            }
            __syncthreads();
        }
        const bool ok = stage_ready<STAGES>(bars, t, &s_abort);
        if (ok) {
            const float *sg = ring + st * BWD3_STAGE_F;
            zp[8] = lds4(&sg[HALO3 + ty * TX + 4 * tx]);
            {
                float2 qp[2];
                lap3_4(qp, sg, zp, tx, ty);
                if (inj) {
                    // each thread reads and clears its own four entries; the
                    // end-of-iteration barrier orders the clear before the
                    // next plane's additions
                    float4 *s4p = reinterpret_cast<float4 *>(&sinj[ty * TX + 4 * tx]);
                    const float4 s4 = *s4p;
                    *s4p = make_float4(0.f, 0.f, 0.f, 0.f);
                    qp[0] = add2(qp[0], lo2(s4));
                    qp[1] = add2(qp[1], hi2(s4));
                }
                const float4 p1 = zp[4];
                const float4 pb4 = lds4(&sg[HALO3 + PT3 + ty * TX + 4 * tx]);
                const float4 c24 = lds4(&sg[HALO3 + 2 * PT3 + ty * TX + 4 * tx]);
                const float4 ia4 = lds4(&sg[HALO3 + 3 * PT3 + ty * TX + 4 * tx]);
                const float4 q4 = lds4(&sg[HALO3 + 4 * PT3 + ty * TX + 4 * tx]);
                float2 pn[2];
#pragma unroll
                for (int h = 0; h < 2; ++h) {
                    const float2 ia2 = half2of(ia4, h);
                    const float2 kb = fma2(ia2, make_float2(2.f, 2.f), make_float2(-1.f, -1.f));
                    const float2 p1h = half2of(p1, h);
                    pn[h] = add2(p1h, fma2(mul2(half2of(c24, h), ia2), qp[h], mul2(kb, sub2(p1h, half2of(pb4, h)))));
                }
                if (rowok && j0 < L.nxp) {
                    const long long so = (long long)it.s * L.fstride;
                    const float o[4] = {pn[0].x, pn[0].y, pn[1].x, pn[1].y};
                    store4(a.pb + so + fidx3(L, i, k0, j0), j0, L.nxp, o);
                    // imaging: G += psi^m (Lhat u^{m-1} + f delta_s / dx), padded grid
                    const float g[4] = {pn[0].x * q4.x, pn[0].y * q4.y, pn[1].x * q4.z, pn[1].y * q4.w};
                    const long long rowb = ((long long)i * L.nyp + k0) * L.nxp;
                    if ((L.nxp & 3) == 0 && j0 + 3 < L.nxp) {
                        red_add4(a.acc_grad + rowb + j0, g[0], g[1], g[2], g[3]);
                    } else {
#pragma unroll
                        for (int p = 0; p < 4; ++p)
                            if (j0 + p < L.nxp) atomicAdd(a.acc_grad + rowb + j0 + p, g[p]);
                    }
                }
            }
        }
#pragma unroll
        for (int z = 0; z < 8; ++z) zp[z] = zp[z + 1];
        __syncthreads();
        if (s_abort) {
            if (threadIdx.x == 0) {
                atomicOr(c.status, ST_TIMEOUT);
                for (int j = t; j < t + STAGES; ++j) mbar_wait(smem_u32(&bars[j % STAGES]), (j / STAGES) & 1, 200000000ull);
            }
            return;
        }
        if (++zi == zend) ++slot;
    }
}

// Compiled variants of each step (index 0 is the default; fwi_autotune may
// pick another per problem shape): ring stages and minimum resident CTAs per
// SM (the register cap). Forward: 3 stages at 4 CTAs per SM, 3 or 2 stages
// at 5 (96 registers); backward: 3 stages at 3 CTAs per SM (shared memory
// allows no more), 2 stages at 4 (128 registers).
struct Variant3 {
    int smem;
    const void *fn;
    int occ;          // resident CTAs per SM (occupancy calculator)
    const void *fn_q; // forward step: the instance that also stores q^n
};

// --------------------------------------------------------- offset Hessian
// The offset-Hessian diagonal of one 3-D time level (Sec. 3, horizontal
// offsets along x): acc[h][i][k][j] += sum_s u_s^n(x + h e_x) u_s^n(x - h e_x),
// h = 0..hmax, at the physical points; u = 0 outside the padded grid (the
// ghost columns, at least 16 on each side, are never written). One launch
// sums up to two levels (u0, u1; a null pointer is skipped): the forward
// step of an even level n leaves u^n and u^{n+1} in its two buffers, so the
// sums of both go out in one pass over the accumulators, whose read and
// write per launch (hmax + 1 planes of the model) would otherwise outweigh
// the fields of a few shots.
// The physical grid is taken as nz ny rows of nx points. A CTA owns 8
// consecutive rows x 64 columns: it copies the rows of SPS shots, with 12
// columns on each side, into shared memory by cp.async (16-byte pieces when
// the sponge width is a multiple of 4, else 4-byte ones), all shots' copies
// in flight together, then each thread forms the products of its 4 points of
// one row from its x window, with its NHC x 4 sums in registers across the
// shots, and adds them with one reduction per offset (a vector one when the
// row of 4 starts on a 16-byte boundary).
constexpr int OH3_W = HMAX_LIMIT;          // staged columns on each side of the tile
constexpr int OH3_RW = TX + 2 * OH3_W;     // floats of one staged row
constexpr int OH3_NP = 8 * (OH3_RW / 4);   // 16-byte pieces of one shot's 8 rows
constexpr int OH3_SPS = 4;                 // shots staged per pass

__device__ __forceinline__ void oh3_cp16(void *dst, const void *src)
{
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(smem_u32(dst)), "l"(src) : "memory");
}
__device__ __forceinline__ void oh3_cp4(void *dst, const void *src)
{
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(smem_u32(dst)), "l"(src) : "memory");
}

template <int NHC>
__global__ void __launch_bounds__(TPB) k_offh3d_level(const float *__restrict__ u0, const float *__restrict__ u1,
                                                      const Lay3D L, int ns, int hmax, float *__restrict__ acc)
{
    static_assert(NHC - 1 <= OH3_W, "window wider than the staged columns");
    static_assert(OH3_NP <= 2 * TPB, "two pieces per thread and shot");
    __shared__ __align__(16) float sm[OH3_SPS][8 * OH3_RW];
    const long long nrow = (long long)L.nz * L.ny;
    const int ntx = (L.nx + TX - 1) / TX;
    const long long r0 = (long long)(blockIdx.x / ntx) * 8;
    const int x0 = (int)(blockIdx.x % ntx) * TX;
    const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
    const bool al = (L.P & 3) == 0;
    // this thread's two pieces: row r of the tile, columns x0 - W + 4 c4 ..;
    // pieces of rows past the grid or wholly right of nx + W are not copied
    // (only points outside the model, never stored, read them)
    long long g[2] = {-1, -1};
    int d[2] = {0, 0};
#pragma unroll
    for (int e2 = 0; e2 < 2; ++e2) {
        const int e = threadIdx.x + e2 * TPB;
        if (e >= OH3_NP) break;
        const int r = e / (OH3_RW / 4), c4 = e - r * (OH3_RW / 4), col = x0 - OH3_W + 4 * c4;
        if (r0 + r < nrow && col < L.nx + OH3_W) {
            const int i = (int)((r0 + r) / L.ny), k = (int)(r0 + r - (long long)i * L.ny);
            g[e2] = fidx3(L, i + L.P, k + L.P, col + L.P);
            d[e2] = r * OH3_RW + 4 * c4;
        }
    }
    float s4[NHC][4];
#pragma unroll
    for (int h = 0; h < NHC; ++h)
#pragma unroll
        for (int p = 0; p < 4; ++p) s4[h][p] = 0.f;
    const int nsb = (ns + OH3_SPS - 1) / OH3_SPS;
#pragma unroll 1
    for (int pass = 0; pass < 2 * nsb; ++pass) {
        // passes over (level, block of OH3_SPS shots): level 0's, then level 1's
        const int l = pass >= nsb, sb = (pass - l * nsb) * OH3_SPS;
        const float *u = l ? u1 : u0;
        if (u == nullptr) continue; // uniform across the CTA
        const int nq = min(OH3_SPS, ns - sb);
        for (int q = 0; q < nq; ++q) {
            const float *src = u + (long long)(sb + q) * L.fstride;
#pragma unroll
            for (int e2 = 0; e2 < 2; ++e2) {
                if (g[e2] < 0) continue;
                if (al) {
                    oh3_cp16(&sm[q][d[e2]], src + g[e2]);
                } else {
#pragma unroll
                    for (int c = 0; c < 4; ++c) oh3_cp4(&sm[q][d[e2] + c], src + g[e2] + c);
                }
            }
        }
        asm volatile("cp.async.commit_group;" ::: "memory");
        asm volatile("cp.async.wait_all;" ::: "memory");
        __syncthreads();
        for (int q = 0; q < nq; ++q) {
            const float *row = &sm[q][ty * OH3_RW + 4 * tx]; // columns x - W .. x + 3 + W
            float w[4 + 2 * OH3_W];
#pragma unroll
            for (int c = 0; c < (4 + 2 * OH3_W) / 4; ++c) {
                const float4 t4 = lds4(row + 4 * c);
                w[4 * c] = t4.x;
                w[4 * c + 1] = t4.y;
                w[4 * c + 2] = t4.z;
                w[4 * c + 3] = t4.w;
            }
#pragma unroll
            for (int h = 0; h < NHC; ++h)
#pragma unroll
                for (int p = 0; p < 4; ++p)
                    s4[h][p] = fmaf(w[OH3_W + p + h], w[OH3_W + p - h], s4[h][p]);
        }
        __syncthreads(); // the next pass overwrites the rows
    }
    const long long row = r0 + ty;
    const int j0 = x0 + 4 * tx;
    if (row >= nrow || j0 >= L.nx) return;
    const long long nphys = nrow * L.nx, o = row * L.nx + j0;
    const bool vec = (L.nx & 3) == 0;
#pragma unroll
    for (int h = 0; h < NHC; ++h) {
        if (h > hmax) break;
        float *dst = acc + h * nphys + o;
        if (vec) {
            red_add4(dst, s4[h][0], s4[h][1], s4[h][2], s4[h][3]);
        } else {
#pragma unroll
            for (int p = 0; p < 4; ++p)
                if (j0 + p < L.nx) atomicAdd(dst + p, s4[h][p]);
        }
    }
}
#define V3F(ST, MINB) \
    {256 + (ST) * FWD3_STAGE_F * 4, (const void *)k_fwd3d<ST, MINB, false>, 0, (const void *)k_fwd3d<ST, MINB, true>}
#define V3B(ST, MINB) {256 + (ST) * BWD3_STAGE_F * 4, (const void *)k_bwd3d<ST, MINB>, 0, nullptr}
Variant3 g_var3f[] = {V3F(3, 4), V3F(3, 5), V3F(2, 5)};
Variant3 g_var3b[] = {V3B(3, 3), V3B(2, 4), V3B(3, 4), V3B(2, 5)};
constexpr int NV3F = (int)(sizeof g_var3f / sizeof g_var3f[0]);
constexpr int NV3B = (int)(sizeof g_var3b / sizeof g_var3b[0]);

Variant3 &variant3(bool backward, int v) { return backward ? g_var3b[v] : g_var3f[v]; }

std::once_flag g_prep3_once;

void prepare_kernels3()
{
    std::call_once(g_prep3_once, [] {
        int dev = 0;
        const bool have_dev = cudaGetDevice(&dev) == cudaSuccess;
        for (int b = 0; b < 2; ++b)
            for (int i = 0; i < (b ? NV3B : NV3F); ++i) {
                Variant3 &v = variant3(b != 0, i);
                int occ = 0;
                if (have_dev) {
                    cudaFuncSetAttribute(v.fn, cudaFuncAttributeMaxDynamicSharedMemorySize, v.smem);
                    if (v.fn_q) cudaFuncSetAttribute(v.fn_q, cudaFuncAttributeMaxDynamicSharedMemorySize, v.smem);
                    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, v.fn, TPB, v.smem) != cudaSuccess)
                        occ = 0;
                }
                v.occ = occ > 0 ? occ : 2;
            }
        cudaGetLastError();
    });
}

// variants kept by the autotuner per (step, padded shape, shots of a group)
struct TuneKey3 {
    bool backward;
    int nzp, nyp, nxp, ns;
    bool operator<(const TuneKey3 &o) const
    {
        return std::tie(backward, nzp, nyp, nxp, ns) < std::tie(o.backward, o.nzp, o.nyp, o.nxp, o.ns);
    }
};
std::mutex g_tune3_mu;
std::map<TuneKey3, std::pair<int, int>> g_tuned3; // (variant, z-segments; 0: chosen per launch shape)

int sm_count3()
{
    int dev = 0, v = 0;
    if (cudaGetDevice(&dev) == cudaSuccess && cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev) == cudaSuccess &&
        v > 0)
        return v;
    cudaGetLastError();
    return 152;
}
} // namespace

int step3_variants(bool backward) { return backward ? NV3B : NV3F; }

int step3_variant_for(const Lay3D &L, int ns, bool backward)
{
    std::lock_guard<std::mutex> lock(g_tune3_mu);
    auto it = g_tuned3.find(TuneKey3{backward, L.nzp, L.nyp, L.nxp, ns});
    return it == g_tuned3.end() ? 0 : it->second.first;
}

int step3_segments_for(const Lay3D &L, int ns, bool backward)
{
    std::lock_guard<std::mutex> lock(g_tune3_mu);
    auto it = g_tuned3.find(TuneKey3{backward, L.nzp, L.nyp, L.nxp, ns});
    return it == g_tuned3.end() ? 0 : it->second.second;
}

void step3_tuned_store(const Lay3D &L, int ns, bool backward, int variant, int nseg)
{
    std::lock_guard<std::mutex> lock(g_tune3_mu);
    g_tuned3[TuneKey3{backward, L.nzp, L.nyp, L.nxp, ns}] = {variant, nseg};
}

void step3_tuned_clear()
{
    std::lock_guard<std::mutex> lock(g_tune3_mu);
    g_tuned3.clear();
}

// z-segments per column for `per` items (columns x shots) of a launch with
// `slots` resident CTAs: the count whose rounds of items, times the planes
// of one item (+2 for the window loads that start a segment), are fewest;
// segments of at least 16 planes, and a smaller count unless 2% shorter.
// A column's items are long (every plane of it), so with few items per slot
// the last round leaves many SMs idle: 200 x 400 x 400 padded to
// 240 x 440 x 440 in groups of 4 shots has 1540 columns x shots for 608
// slots (2.53 rounds: 3 x 242 planes), cut in 3 segments 7.6 rounds (8 x
// 82 planes).
int pick_segments(int nzp, long long per, long long slots)
{
    int best = 1;
    double best_cost = 1e300;
    for (int k = 1; k <= 8; ++k) {
        const int segl = (nzp + k - 1) / k;
        if (k > 1 && segl < 16) break;
        if ((nzp + segl - 1) / segl != k) continue; // the same cut as a smaller count
        const long long rounds = (per * k + slots - 1) / slots;
        const double cost = (double)rounds * (segl + 2);
        if (cost < 0.98 * best_cost) {
            best_cost = cost;
            best = k;
        }
    }
    return best;
}

Tiling3 make_tiling3(const Lay3D &L, int ns, bool backward, int variant, int nseg)
{
    prepare_kernels3();
    if (variant < 0 || variant >= step3_variants(backward)) variant = 0;
    Tiling3 t;
    t.nty = (L.nyp + TY3 - 1) / TY3;
    t.ntx = (L.nxp + TX - 1) / TX;
    const long long per = (long long)t.nty * t.ntx * ns;
    const long long slots = (long long)sm_count3() * variant3(backward, variant).occ;
    if (nseg <= 0) nseg = pick_segments(L.nzp, per, slots);
    nseg = std::min(nseg, L.nzp);
    t.segl = (L.nzp + nseg - 1) / nseg;
    t.nseg = (L.nzp + t.segl - 1) / t.segl;
    const long long items = per * t.nseg;
    t.ctas = (int)(items < slots ? items : slots);
    return t;
}

namespace {
template <class A>
cudaError_t launch3(const void *fn, const Variant3 &v, const A &a, const Tiling3 &t, cudaStream_t st)
{
    if (t.ctas <= 0) return cudaSuccess;
    void *args[] = {const_cast<A *>(&a)};
    return cudaLaunchKernel(fn, dim3(t.ctas), dim3(TPB), args, v.smem, st);
}
} // namespace

cudaError_t launch_fwd3d(const Fwd3Args &a, const Tiling3 &t, int variant, cudaStream_t st)
{
    if (variant < 0 || variant >= NV3F) return cudaErrorInvalidValue;
    if (a.uout == nullptr && a.qout == nullptr) return cudaErrorInvalidValue;
    const Variant3 &v = g_var3f[variant];
    return launch3(a.qout != nullptr ? v.fn_q : v.fn, v, a, t, st);
}

cudaError_t launch_bwd3d(const Bwd3Args &a, const Tiling3 &t, int variant, cudaStream_t st)
{
    if (variant < 0 || variant >= NV3B) return cudaErrorInvalidValue;
    const Variant3 &v = g_var3b[variant];
    return launch3(v.fn, v, a, t, st);
}

cudaError_t launch_offh3d(const float *u0, const float *u1, const Lay3D &L, int ns, int hmax, float *acc,
                          cudaStream_t st)
{
    if (hmax < 0 || hmax > HMAX_LIMIT || ns < 0 || !acc) return cudaErrorInvalidValue;
    const long long tiles = ((long long)L.nz * L.ny + 7) / 8 * ((L.nx + TX - 1) / TX);
    if (tiles == 0 || ns == 0 || (!u0 && !u1)) return cudaSuccess;
    if (tiles > 0x7fffffffLL) return cudaErrorInvalidValue;
    const unsigned blocks = (unsigned)tiles;
    // compiled offset counts: 4 (hmax <= 3), 11 (<= 10), 13 (<= 12)
    if (hmax <= 3)
        k_offh3d_level<4><<<blocks, TPB, 0, st>>>(u0, u1, L, ns, hmax, acc);
    else if (hmax <= 10)
        k_offh3d_level<11><<<blocks, TPB, 0, st>>>(u0, u1, L, ns, hmax, acc);
    else
        k_offh3d_level<13><<<blocks, TPB, 0, st>>>(u0, u1, L, ns, hmax, acc);
    return cudaGetLastError();
}

bool encode_field_map3(CUtensorMap *map, const float *base, const Lay3D &L, int nfields, int bx, int by)
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
    const cuuint64_t dims[4] = {(cuuint64_t)L.pitch, (cuuint64_t)L.rows, (cuuint64_t)L.planes, (cuuint64_t)nfields};
    const cuuint64_t strides[3] = {(cuuint64_t)L.pitch * sizeof(float), (cuuint64_t)L.plane * sizeof(float),
                                   (cuuint64_t)L.fstride * sizeof(float)};
    const cuuint32_t box[4] = {(cuuint32_t)bx, (cuuint32_t)by, 1, 1};
    const cuuint32_t estr[4] = {1, 1, 1, 1};
    CUresult r = encode(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 4, const_cast<float *>(base), dims, strides, box,
                        estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                        CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS;
}

} // namespace fwi
