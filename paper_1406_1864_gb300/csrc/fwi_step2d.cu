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
//     u^{m-2} = 2 u^{m-1} + c2 q^{m-1} - u^m, the sponge cells restored from
//     the checkpoint (leapfrog is time-reversible where eta = 0),
//   - zero-lag imaging [Sec. 2]: G += psi^m * q^{m-1}, q = Lhat u + f delta_s,
//     which is dx^2 (L u + s); the factor 2 / (v dx^2) is applied once at the
//     end (fwi_aux.cu).
//
// Work decomposition: a CTA of 128 threads owns a 64 x (8 RZ) tile of the
// padded grid and a group of shots; it loops over its shots, staging each
// shot's tile (plus a stencil halo) in shared memory with 16-byte loads, so
// the accumulators of its tile (illumination, offset Hessian, gradient) stay in
// registers across the shot loop and are written once per step per group.
// Each thread owns a float4 of 4 columns on RZ rows.
#include "fwi_internal.h"

namespace fwi {

#ifndef FWD_MINB
#define FWD_MINB 4
#endif
#ifndef BWD_MINB
#define BWD_MINB 3
#endif

namespace {

// 8th-order centred second-derivative weights
constexpr float W0 = -205.0f / 72.0f;
constexpr float W1 = 8.0f / 5.0f;
constexpr float W2 = -1.0f / 5.0f;
constexpr float W3 = 8.0f / 315.0f;
constexpr float W4 = -1.0f / 560.0f;

// Lhat u at one point from the symmetric neighbour sums
// s_k = (x_{-k} + x_{+k}) + (z_{-k} + z_{+k}). The forward and the backward
// kernels both call this, so q is bitwise the same in both passes.
__device__ __forceinline__ float lap8(float c, float s1, float s2, float s3, float s4)
{
    float q = (2.0f * W0) * c;
    q = fmaf(W1, s1, q);
    q = fmaf(W2, s2, q);
    q = fmaf(W3, s3, q);
    q = fmaf(W4, s4, q);
    return q;
}

__device__ __forceinline__ float comp(const float4 &v, int p)
{
    return p == 0 ? v.x : (p == 1 ? v.y : (p == 2 ? v.z : v.w));
}

__device__ __forceinline__ float4 lds4(const float *p) { return *reinterpret_cast<const float4 *>(p); }

__device__ __forceinline__ float4 ldg4(const float *p) { return __ldg(reinterpret_cast<const float4 *>(p)); }

// sponge coefficients at padded cell (i, j): 1/(1 + eta dt) and 1 - eta dt;
// exactly 1 and 1 in the model.
__device__ __forceinline__ void sponge_coef(const Lay2D &L, int i, int j, float &ia, float &b,
                                            bool &in_sponge)
{
    const int dz = sponge_depth(i, L.P, L.nz);
    const int dxs = sponge_depth(j, L.P, L.nx);
    in_sponge = (dz | dxs) != 0;
    ia = 1.0f;
    b = 1.0f;
    if (in_sponge) {
        const float e = L.etamax_dt * (float)(dz * dz + dxs * dxs) * L.inv_p2;
        ia = __fdiv_rn(1.0f, 1.0f + e);
        b = 1.0f - e;
    }
}

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

// Cooperative load of a (TZ + 8) x (TX + 2 HX) tile of one field into shared
// memory. Rows/columns that no valid output needs are filled with zeros
// instead of being read.
template <int TZ, int HX>
__device__ __forceinline__ void load_tile(float *sm, const float *f, const Lay2D &L, int bi, int bj)
{
    constexpr int TXS = TX + 2 * HX;
    constexpr int NV = TXS / 4;
    constexpr int NR = TZ + 2 * RADIUS;
    for (int e = threadIdx.x; e < NR * NV; e += TPB) {
        const int r = e / NV;
        const int v = e - r * NV;
        const int gi = bi - RADIUS + r;
        const int gj = bj - HX + 4 * v;
        float4 val = make_float4(0.f, 0.f, 0.f, 0.f);
        if (gi < L.nzp + RADIUS && gj < L.nxp + HX) val = ldg4(f + fidx(L, gi, gj));
        *reinterpret_cast<float4 *>(&sm[r * TXS + 4 * v]) = val;
    }
}

} // namespace

// ------------------------------------------------------------ forward step
template <int RZ, int HX, bool WITH_H>
__global__ void __launch_bounds__(TPB, WITH_H ? 3 : FWD_MINB) k_fwd_step(const FwdArgs a)
{
    constexpr int TZ = 8 * RZ;
    constexpr int TXS = TX + 2 * HX;
    constexpr int NH = WITH_H ? HMAX_LIMIT + 1 : 1;
    static_assert(!WITH_H || (RZ == 1 && HX == 12), "offset Hessian uses RZ=1, HX=12");
    __shared__ __align__(16) float sm[(TZ + 2 * RADIUS) * TXS];

    const StepCommon &c = a.c;
    const Lay2D &L = c.L;
    const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
    const int bi = blockIdx.y * TZ, bj = blockIdx.x * TX;
    const int i0 = bi + ty * RZ, j0 = bj + 4 * tx;
    const int tile = blockIdx.y * c.ntx + blockIdx.x;
    const int s0 = blockIdx.z * c.spg;
    const int s1 = min(c.ns, s0 + c.spg);
    const bool colok = j0 < L.nxp;
    const bool do_illum = a.acc_illum != nullptr;

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

    for (int s = s0; s < s1; ++s) {
        const float *uc = a.ucur + (long long)s * L.fstride;
        float *up = a.uprev + (long long)s * L.fstride;
        // u^{n-1} of this thread's points, in flight during the tile load
        float4 um1[RZ];
#pragma unroll
        for (int r = 0; r < RZ; ++r) {
            um1[r] = make_float4(0.f, 0.f, 0.f, 0.f);
            if (!a.last && colok && i0 + r < L.nzp)
                um1[r] = __ldcs(reinterpret_cast<const float4 *>(up + fidx(L, i0 + r, j0)));
        }
        load_tile<TZ, HX>(sm, uc, L, bi, bj);
        const int src_off = c.src_off[s];
        const float src_amp = a.last ? 0.f : c.wav[(long long)s * c.nt + a.n] * c.src_scale;
        __syncthreads();

        // receiver extraction d^n = R u^n
        if (a.seis != nullptr) {
            const int rb = a.rt.ptr[tile * c.ns + s], re = a.rt.ptr[tile * c.ns + s + 1];
            for (int e = rb + (int)threadIdx.x; e < re; e += TPB) {
                const int2 en = a.rt.ent[e];
                const int zl = en.x / TX, xl = en.x - zl * TX;
                a.seis[((long long)s * c.nt + a.n) * c.nrec + en.y] =
                    sm[(zl + RADIUS) * TXS + HX + xl];
            }
        }

        // column window rows -4 .. RZ+3 around this thread's rows
        float4 zc[RZ + 2 * RADIUS];
#pragma unroll
        for (int k = 0; k < RZ + 2 * RADIUS; ++k) zc[k] = lds4(&sm[(ty * RZ + k) * TXS + HX + 4 * tx]);

#pragma unroll
        for (int r = 0; r < RZ; ++r) {
            const int i = i0 + r;
            const float *row = &sm[(ty * RZ + r + RADIUS) * TXS + HX + 4 * tx];
            constexpr int WL = WITH_H ? HMAX_LIMIT : RADIUS; // window left extent
            constexpr int NW = (2 * WL + 4) / 4;             // float4s in the window
            float w[4 * NW];
#pragma unroll
            for (int k = 0; k < NW; ++k) {
                const float4 t = lds4(row - WL + 4 * k);
                w[4 * k] = t.x; w[4 * k + 1] = t.y; w[4 * k + 2] = t.z; w[4 * k + 3] = t.w;
            }
            float out[4];
#pragma unroll
            for (int p = 0; p < 4; ++p) {
                const int j = j0 + p;
                const float u0 = w[WL + p];
                float um = comp(um1[r], p);
                out[p] = 0.f;
                if (!a.last) {
                    const float s1v = (w[WL + p - 1] + w[WL + p + 1]) + (comp(zc[r + 3], p) + comp(zc[r + 5], p));
                    const float s2v = (w[WL + p - 2] + w[WL + p + 2]) + (comp(zc[r + 2], p) + comp(zc[r + 6], p));
                    const float s3v = (w[WL + p - 3] + w[WL + p + 3]) + (comp(zc[r + 1], p) + comp(zc[r + 7], p));
                    const float s4v = (w[WL + p - 4] + w[WL + p + 4]) + (comp(zc[r + 0], p) + comp(zc[r + 8], p));
                    float q = lap8(u0, s1v, s2v, s3v, s4v);
                    if (fidx(L, i, j) == src_off) q += src_amp;
                    if (i < L.nzp && j < L.nxp) {
                        const float c2v = __ldg(c.c2 + fidx(L, i, j));
                        float ia, b;
                        bool sp;
                        sponge_coef(L, i, j, ia, b, sp);
                        const float T = fmaf(c2v, q, 2.0f * u0);
                        const float un = fmaf(-b, um, T) * ia;
                        out[p] = un;
                        if (sp && a.band != nullptr)
                            a.band[((long long)s * c.nt + a.n + 1) * L.nband + band_index(L, i, j)] = un;
                        if (a.illum_utt) {
                            const float d2 = (un - 2.0f * u0) + um;
                            acc_i[r][p] = fmaf(d2, d2, acc_i[r][p]);
                        }
                    }
                }
                if (!a.illum_utt) acc_i[r][p] = fmaf(u0, u0, acc_i[r][p]);
                if (WITH_H) {
#pragma unroll
                    for (int h = 0; h < NH; ++h)
                        if (h <= a.hmax) acc_h[h][p] = fmaf(w[WL + p + h], w[WL + p - h], acc_h[h][p]);
                }
            }
            if (!a.last && colok && i < L.nzp) store4(up + fidx(L, i, j0), j0, L.nxp, out);
        }
        __syncthreads();
    }

    // flush this group's accumulators (physical cells only)
    const long long nphys = (long long)L.nz * L.nx;
#pragma unroll
    for (int r = 0; r < RZ; ++r) {
        const int iz = i0 + r - L.P;
        if (iz < 0 || iz >= L.nz) continue;
#pragma unroll
        for (int p = 0; p < 4; ++p) {
            const int ix = j0 + p - L.P;
            if (ix < 0 || ix >= L.nx) continue;
            const long long o = (long long)iz * L.nx + ix;
            if (do_illum) a.acc_illum[blockIdx.z * nphys + o] += acc_i[r][p];
            if (WITH_H) {
#pragma unroll
                for (int h = 0; h < NH; ++h)
                    if (h <= a.hmax)
                        a.acc_offh[((long long)blockIdx.z * (a.hmax + 1) + h) * nphys + o] += acc_h[h][p];
            }
        }
    }
}

// ----------------------------------------------------------- backward step
template <int RZ>
__global__ void __launch_bounds__(TPB, BWD_MINB) k_bwd_step(const BwdArgs a)
{
    constexpr int TZ = 8 * RZ;
    constexpr int HX = RADIUS;
    constexpr int TXS = TX + 2 * HX;
    __shared__ __align__(16) float su[(TZ + 2 * RADIUS) * TXS];
    __shared__ __align__(16) float sp[(TZ + 2 * RADIUS) * TXS];
    __shared__ float sinj[TZ * TX];

    const StepCommon &c = a.c;
    const Lay2D &L = c.L;
    const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
    const int bi = blockIdx.y * TZ, bj = blockIdx.x * TX;
    const int i0 = bi + ty * RZ, j0 = bj + 4 * tx;
    const int tile = blockIdx.y * c.ntx + blockIdx.x;
    const int s0 = blockIdx.z * c.spg;
    const int s1 = min(c.ns, s0 + c.spg);
    const bool colok = j0 < L.nxp;
    const int m = a.m;

    for (int e = threadIdx.x; e < TZ * TX; e += TPB) sinj[e] = 0.f;

    float acc_g[RZ][4];
#pragma unroll
    for (int r = 0; r < RZ; ++r)
#pragma unroll
        for (int p = 0; p < 4; ++p) acc_g[r][p] = 0.f;

    for (int s = s0; s < s1; ++s) {
        const long long so = (long long)s * L.fstride;
        float4 uam[RZ], pbm[RZ];
#pragma unroll
        for (int r = 0; r < RZ; ++r) {
            uam[r] = make_float4(0.f, 0.f, 0.f, 0.f);
            pbm[r] = make_float4(0.f, 0.f, 0.f, 0.f);
            if (colok && i0 + r < L.nzp) {
                pbm[r] = __ldcs(reinterpret_cast<const float4 *>(a.pb + so + fidx(L, i0 + r, j0)));
                if (m >= 2) uam[r] = __ldcs(reinterpret_cast<const float4 *>(a.ua + so + fidx(L, i0 + r, j0)));
            }
        }
        load_tile<TZ, HX>(su, a.ub + so, L, bi, bj);
        load_tile<TZ, HX>(sp, a.pa + so, L, bi, bj);
        const int rb = a.rt.ptr[tile * c.ns + s], re = a.rt.ptr[tile * c.ns + s + 1];
        const bool has_rec = rb < re;
        for (int e = rb + (int)threadIdx.x; e < re; e += TPB) {
            const int2 en = a.rt.ent[e];
            atomicAdd(&sinj[en.x], a.adj[((long long)s * c.nt + m) * c.nrec + en.y] * a.adj_scale);
        }
        const int src_off = c.src_off[s];
        const float src_amp = c.wav[(long long)s * c.nt + (m - 1)] * c.src_scale;
        __syncthreads();

        float4 zu[RZ + 2 * RADIUS], zp[RZ + 2 * RADIUS];
#pragma unroll
        for (int k = 0; k < RZ + 2 * RADIUS; ++k) {
            zu[k] = lds4(&su[(ty * RZ + k) * TXS + HX + 4 * tx]);
            zp[k] = lds4(&sp[(ty * RZ + k) * TXS + HX + 4 * tx]);
        }
#pragma unroll
        for (int r = 0; r < RZ; ++r) {
            const int i = i0 + r;
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
            float unew[4], pnew[4];
#pragma unroll
            for (int p = 0; p < 4; ++p) {
                const int j = j0 + p;
                unew[p] = 0.f;
                pnew[p] = 0.f;
                // q^{m-1} = Lhat u^{m-1} + f(t_{m-1}) delta_s (as in the forward step m-1)
                const float u1 = wu[4 + p];
                float qu = lap8(u1,
                                (wu[3 + p] + wu[5 + p]) + (comp(zu[r + 3], p) + comp(zu[r + 5], p)),
                                (wu[2 + p] + wu[6 + p]) + (comp(zu[r + 2], p) + comp(zu[r + 6], p)),
                                (wu[1 + p] + wu[7 + p]) + (comp(zu[r + 1], p) + comp(zu[r + 7], p)),
                                (wu[0 + p] + wu[8 + p]) + (comp(zu[r + 0], p) + comp(zu[r + 8], p)));
                if (fidx(L, i, j) == src_off) qu += src_amp;
                const float p1 = wp[4 + p];
                float qp = lap8(p1,
                                (wp[3 + p] + wp[5 + p]) + (comp(zp[r + 3], p) + comp(zp[r + 5], p)),
                                (wp[2 + p] + wp[6 + p]) + (comp(zp[r + 2], p) + comp(zp[r + 6], p)),
                                (wp[1 + p] + wp[7 + p]) + (comp(zp[r + 1], p) + comp(zp[r + 7], p)),
                                (wp[0 + p] + wp[8 + p]) + (comp(zp[r + 0], p) + comp(zp[r + 8], p)));
                if (has_rec) qp += sinj[(ty * RZ + r) * TX + 4 * tx + p];
                if (i < L.nzp && j < L.nxp) {
                    const float c2v = __ldg(c.c2 + fidx(L, i, j));
                    float ia, b;
                    bool spg;
                    sponge_coef(L, i, j, ia, b, spg);
                    const float ps = fmaf(-b, comp(pbm[r], p), fmaf(c2v, qp, 2.0f * p1)) * ia;
                    pnew[p] = ps;
                    acc_g[r][p] = fmaf(ps, qu, acc_g[r][p]);
                    if (m >= 2) {
                        if (spg) {
                            unew[p] = (m - 2 >= 1)
                                          ? __ldcs(a.band + ((long long)s * c.nt + (m - 2)) * L.nband + band_index(L, i, j))
                                          : 0.f;
                        } else {
                            unew[p] = fmaf(c2v, qu, 2.0f * u1) - comp(uam[r], p);
                        }
                    }
                }
            }
            if (colok && i < L.nzp) {
                store4(a.pb + so + fidx(L, i, j0), j0, L.nxp, pnew);
                if (m >= 2) store4(a.ua + so + fidx(L, i, j0), j0, L.nxp, unew);
            }
        }
        __syncthreads();
        if (has_rec) {
            for (int e = rb + (int)threadIdx.x; e < re; e += TPB) sinj[a.rt.ent[e].x] = 0.f;
            __syncthreads();
        }
    }

    // flush this group's gradient sum (padded grid)
#pragma unroll
    for (int r = 0; r < RZ; ++r) {
        const int i = i0 + r;
        if (i >= L.nzp) continue;
#pragma unroll
        for (int p = 0; p < 4; ++p) {
            const int j = j0 + p;
            if (j >= L.nxp) continue;
            a.acc_grad[((long long)blockIdx.z * L.nzp + i) * L.nxp + j] += acc_g[r][p];
        }
    }
}

// ---------------------------------------------------------------- launchers
namespace {
constexpr int FWD_RZ = 4;
constexpr int BWD_RZ = 2;
}

Tiling make_tiling(const Lay2D &L, int ns, int tz, int target_ctas)
{
    Tiling t;
    t.tz = tz;
    t.ntx = (L.nxp + TX - 1) / TX;
    t.ntz = (L.nzp + tz - 1) / tz;
    const int tiles = t.ntx * t.ntz;
    int g = (target_ctas + tiles / 2) / tiles;
    if (g < 1) g = 1;
    if (g > ns) g = ns;
    t.spg = (ns + g - 1) / g;
    t.groups = (ns + t.spg - 1) / t.spg;
    return t;
}

int fwd_tile_height(bool with_offh) { return with_offh ? 8 : 8 * FWD_RZ; }
int bwd_tile_height() { return 8 * BWD_RZ; }

cudaError_t launch_fwd_step(const FwdArgs &a, const Tiling &t, bool with_offh, cudaStream_t st)
{
    dim3 grid(t.ntx, t.ntz, t.groups);
    if (with_offh)
        k_fwd_step<1, HMAX_LIMIT, true><<<grid, TPB, 0, st>>>(a);
    else
        k_fwd_step<FWD_RZ, RADIUS, false><<<grid, TPB, 0, st>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_bwd_step(const BwdArgs &a, const Tiling &t, cudaStream_t st)
{
    dim3 grid(t.ntx, t.ntz, t.groups);
    k_bwd_step<BWD_RZ><<<grid, TPB, 0, st>>>(a);
    return cudaGetLastError();
}

int occupancy_fwd(bool with_offh)
{
    int n = 0;
    if (with_offh)
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_fwd_step<1, HMAX_LIMIT, true>, TPB, 0);
    else
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_fwd_step<FWD_RZ, RADIUS, false>, TPB, 0);
    return n;
}

int occupancy_bwd()
{
    int n = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_bwd_step<BWD_RZ>, TPB, 0);
    return n;
}

} // namespace fwi
