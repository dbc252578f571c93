// fwi_aux.cu -- the small kernels around the time loops (sm_103a):
// model preparation, misfits and adjoint sources (OLS of Sec. 2 and the
// time-integral misfit of Eq. 2), folding of the padded-grid gradient,
// illumination / offset-Hessian outputs (Eq. 1, Sec. 3) and the diagonal
// preconditioning g / (P + eps max P) of Sec. 3.1.
#include "fwi_device.cuh"
#include "fwi_internal.h"

#include <cfloat>
#include <cuda_bf16.h>
#include <cuda_fp16.h>

namespace fwi {

namespace {

constexpr int NT1 = 256;

__device__ __forceinline__ double warp_sum(double v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// sum of v over the block, added atomically to *out (FP64)
__device__ __forceinline__ void block_sum_add(double v, double *out)
{
    __shared__ double part[NT1 / 32];
    v = warp_sum(v);
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    if (lane == 0) part[wid] = v;
    __syncthreads();
    if (wid == 0) {
        v = lane < NT1 / 32 ? part[lane] : 0.0;
        v = warp_sum(v);
        if (lane == 0) atomicAdd(out, v);
    }
}

__device__ __forceinline__ int clampi(int a, int lo, int hi) { return a < lo ? lo : (a > hi ? hi : a); }

// c2 = (v dt / dx)^2 on the padded grid, the sponge replicating the nearest
// model cell; checks v > 0, finite, and the stability limit.
// c2 = (v dt/dx)^2 and the sponge factor 1 / (1 + eta dt) of every padded
// cell, eta dt = eta_max dt (d_z^2 + d_x^2) / P^2 with d the depth into the
// sponge (the two parts summed in FP32, then one correctly rounded division)
__global__ void k_prep_c2(const Lay2D L, const float *__restrict__ v, float *__restrict__ c2,
                          float *__restrict__ damp, float cfl_limit, int *status)
{
    const long long n = (long long)L.nzp * L.nxp;
    int bad = 0;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n;
         e += (long long)gridDim.x * blockDim.x) {
        const int i = (int)(e / L.nxp), j = (int)(e - (long long)i * L.nxp);
        const int iz = clampi(i - L.P, 0, L.nz - 1), ix = clampi(j - L.P, 0, L.nx - 1);
        const float vv = v[(long long)iz * L.nx + ix];
        const float r = vv * L.dt / L.dx;
        if (!(vv > 0.f) || !isfinite(vv)) bad |= ST_BAD_VELOCITY;
        else if (r > cfl_limit) bad |= ST_CFL;
        c2[fidx(L, i, j)] = r * r;
        const int dz = sponge_depth(i, L.P, L.nz), dxs = sponge_depth(j, L.P, L.nx);
        const float ez = L.etamax_dt * (float)(dz * dz) * L.inv_p2;
        const float ex = L.etamax_dt * (float)(dxs * dxs) * L.inv_p2;
        damp[fidx(L, i, j)] = 1.0f / (1.0f + (ez + ex));
    }
    if (bad) atomicOr(status, bad);
}

// dc2 = 2 c2 dv / v on the padded grid (dv edge-replicated like v): the
// derivative of c2 = (v dt/dx)^2 along dv
__global__ void k_prep_dc2(const Lay2D L, const float *__restrict__ v, const float *__restrict__ dv,
                           const float *__restrict__ c2, float *__restrict__ dc2)
{
    const long long n = (long long)L.nzp * L.nxp;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n;
         e += (long long)gridDim.x * blockDim.x) {
        const int i = (int)(e / L.nxp), j = (int)(e - (long long)i * L.nxp);
        const long long m = (long long)clampi(i - L.P, 0, L.nz - 1) * L.nx + clampi(j - L.P, 0, L.nx - 1);
        const long long o = fidx(L, i, j);
        // dv times a factor that does not depend on dv (correctly rounded
        // quotient), so that dc2 scales exactly with dv
        dc2[o] = dv[m] * __fdiv_rn(2.0f * c2[o], v[m]);
    }
}

// D~(y, h) = 2 c2(y + h) dv(y + h, h) / v(y + h) for padded y, |h| <= hext
// (dv_ext edge-replicated into the sponge, like v), zero where y + h leaves
// the padded grid and for hext < |h| <= he; planes h = -he..he
__global__ void k_prep_dext(const Lay2D L, const float *__restrict__ v, const float *__restrict__ dv_ext,
                            const float *__restrict__ c2, int hext, int he, float *__restrict__ dext)
{
    const long long npl = (long long)L.nzp * L.nxp;
    const long long n = npl * (2 * he + 1);
    const long long nphys = (long long)L.nz * L.nx;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n;
         e += (long long)gridDim.x * blockDim.x) {
        const int pl = (int)(e / npl);
        const long long r = e - (long long)pl * npl;
        const int i = (int)(r / L.nxp), j = (int)(r - (long long)i * L.nxp);
        const int h = pl - he, jx = j + h;
        float d = 0.f;
        if (h >= -hext && h <= hext && jx >= 0 && jx < L.nxp) {
            const long long m = (long long)clampi(i - L.P, 0, L.nz - 1) * L.nx + clampi(jx - L.P, 0, L.nx - 1);
            d = dv_ext[(long long)(h + hext) * nphys + m] * __fdiv_rn(2.0f * c2[fidx(L, i, jx)], v[m]);
        }
        dext[(long long)pl * L.fstride + fidx(L, i, j)] = d;
    }
}

// image(x, h) = sum over the padded cells x' folding into physical x of
// 2 v(x') / (v(x' - h)^2 dx^2) acc(x' - h, h), |h| <= hext
__global__ void k_fold_ext(const Lay2D L, const float *__restrict__ acc, int he, int hext,
                           const float *__restrict__ v, float *__restrict__ image)
{
    const long long nphys = (long long)L.nz * L.nx;
    const long long n = nphys * (2 * hext + 1);
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n;
         e += (long long)gridDim.x * blockDim.x) {
        const int pl = (int)(e / nphys);
        const long long o = e - (long long)pl * nphys;
        const int h = pl - hext;
        const int iz = (int)(o / L.nx), ix = (int)(o - (long long)iz * L.nx);
        const int ia = iz == 0 ? 0 : iz + L.P, ib = iz == L.nz - 1 ? L.nzp - 1 : iz + L.P;
        const int ja = ix == 0 ? 0 : ix + L.P, jb = ix == L.nx - 1 ? L.nxp - 1 : ix + L.P;
        const float *ap = acc + (long long)(h + he) * L.nzp * L.nxp;
        float sum = 0.f;
        for (int i = ia; i <= ib; ++i)
            for (int j = ja; j <= jb; ++j) {
                const int jy = j - h;
                if (jy < 0 || jy >= L.nxp) continue;
                const float vy = v[(long long)clampi(i - L.P, 0, L.nz - 1) * L.nx + clampi(jy - L.P, 0, L.nx - 1)];
                sum += ap[(long long)i * L.nxp + jy] / (vy * vy);
            }
        image[e] = sum * (2.0f * v[o] / (L.dx * L.dx));
    }
}

// Plessix-Mulder receiver factor of a fixed spread: the integral over the
// receiver line of 1 / distance, asinh((xmax - x)/z) - asinh((xmin - x)/z),
// x = j dx, z = |i - zr| dx floored at dx / 2 (the receiver row itself)
__global__ void k_pm_factor(int nz, int nx, float dx, float xmin, float xmax, float zr, float *__restrict__ out)
{
    const long long n = (long long)nz * nx;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n;
         e += (long long)gridDim.x * blockDim.x) {
        const int i = (int)(e / nx), j = (int)(e - (long long)i * nx);
        const float z = fmaxf(fabsf((float)i - zr) * dx, 0.5f * dx);
        const float x = (float)j * dx;
        out[e] = asinhf((xmax - x) / z) - asinhf((xmin - x) / z);
    }
}

// out += W illum with W the Plessix-Mulder factor of one receiver spread
// (as k_pm_factor)
__global__ void k_pm_accumulate(int nz, int nx, float dx, float xmin, float xmax, float zr,
                                const float *__restrict__ illum, float *__restrict__ out)
{
    const long long n = (long long)nz * nx;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n;
         e += (long long)gridDim.x * blockDim.x) {
        const int i = (int)(e / nx), j = (int)(e - (long long)i * nx);
        const float z = fmaxf(fabsf((float)i - zr) * dx, 0.5f * dx);
        const float x = (float)j * dx;
        out[e] = fmaf(asinhf((xmax - x) / z) - asinhf((xmin - x) / z), illum[e], out[e]);
    }
}

// The bounded wait of the step kernels on an mbarrier that no thread arrives
// at: every lane gives up after limit_ns, and the block raises ST_TIMEOUT as
// a step kernel does (then returns, leaving the context usable)
__global__ void k_wait_selftest(uint64_t limit_ns, int *status)
{
    __shared__ __align__(8) uint64_t bar;
    if (threadIdx.x == 0) {
        mbar_init(smem_u32(&bar), 1);
        fence_mbar_init();
    }
    __syncthreads();
    const bool done = mbar_wait(smem_u32(&bar), 0, limit_ns);
    if (!done && threadIdx.x == 0) atomicOr(status, ST_TIMEOUT);
}

// rows of a [rows][n] array all equal to src[0 .. n-1]
__global__ void k_replicate_row(const float *__restrict__ src, int n, int rows, float *__restrict__ dst)
{
    const long long tot = (long long)rows * n;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < tot;
         e += (long long)gridDim.x * blockDim.x)
        dst[e] = src[e % n];
}

// out[h][x] = scale[h][x] * recv[min(h, rn - 1)][x], h < planes
__global__ void k_scale_product(long long nphys, int planes, const float *__restrict__ scale,
                                const float *__restrict__ recv, int rn, float *__restrict__ out)
{
    const long long n = nphys * planes;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n;
         e += (long long)gridDim.x * blockDim.x) {
        const int h = (int)(e / nphys);
        const long long x = e - (long long)h * nphys;
        out[e] = scale[e] * recv[(long long)min(h, rn - 1) * nphys + x];
    }
}

// 3-D: c2 and the sponge factor of every padded cell (edge-replicated
// velocity; eta dt sums the three axes' parts, as the 2-D kernel does two)
__global__ void k_prep3d(const Lay3D L, const float *__restrict__ v, float *__restrict__ c2,
                         float *__restrict__ damp, float cfl_limit, int *status)
{
    const long long n = (long long)L.nzp * L.nyp * L.nxp;
    int bad = 0;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n;
         e += (long long)gridDim.x * blockDim.x) {
        const int i = (int)(e / ((long long)L.nyp * L.nxp));
        const long long r = e - (long long)i * L.nyp * L.nxp;
        const int k = (int)(r / L.nxp), j = (int)(r - (long long)k * L.nxp);
        const int iz = clampi(i - L.P, 0, L.nz - 1), iy = clampi(k - L.P, 0, L.ny - 1),
                  ix = clampi(j - L.P, 0, L.nx - 1);
        const float vv = v[((long long)iz * L.ny + iy) * L.nx + ix];
        const float rr = vv * L.dt / L.dx;
        if (!(vv > 0.f) || !isfinite(vv)) bad |= ST_BAD_VELOCITY;
        else if (rr > cfl_limit) bad |= ST_CFL;
        const long long o = fidx3(L, i, k, j);
        c2[o] = rr * rr;
        const int dz = sponge_depth(i, L.P, L.nz), dy = sponge_depth(k, L.P, L.ny), dxs = sponge_depth(j, L.P, L.nx);
        const float ez = L.etamax_dt * (float)(dz * dz) * L.inv_p2;
        const float ey = L.etamax_dt * (float)(dy * dy) * L.inv_p2;
        const float ex = L.etamax_dt * (float)(dxs * dxs) * L.inv_p2;
        damp[o] = 1.0f / (1.0f + ((ez + ey) + ex));
    }
    if (bad) atomicOr(status, bad);
}

// 3-D fold of the padded-grid imaging sum into the model cells (each edge
// cell collects the sponge cells that replicate it), times 2/(v dx^2)
__global__ void k_fold_grad3d(const Lay3D L, const float *__restrict__ acc, const float *__restrict__ v,
                              float *__restrict__ grad)
{
    const long long n = (long long)L.nz * L.ny * L.nx;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n;
         e += (long long)gridDim.x * blockDim.x) {
        const int iz = (int)(e / ((long long)L.ny * L.nx));
        const long long r = e - (long long)iz * L.ny * L.nx;
        const int iy = (int)(r / L.nx), ix = (int)(r - (long long)iy * L.nx);
        const int ia = iz == 0 ? 0 : iz + L.P, ib = iz == L.nz - 1 ? L.nzp - 1 : iz + L.P;
        const int ka = iy == 0 ? 0 : iy + L.P, kb = iy == L.ny - 1 ? L.nyp - 1 : iy + L.P;
        const int ja = ix == 0 ? 0 : ix + L.P, jb = ix == L.nx - 1 ? L.nxp - 1 : ix + L.P;
        float sum = 0.f;
        for (int i = ia; i <= ib; ++i)
            for (int k = ka; k <= kb; ++k)
                for (int j = ja; j <= jb; ++j) sum += acc[((long long)i * L.nyp + k) * L.nxp + j];
        grad[e] = sum * (2.0f / (v[e] * L.dx * L.dx));
    }
}

// r = syn - obs (in place in syn), misfit += 1/2 sum r^2 (misfit may be NULL)
__global__ void k_residual_ols(float *__restrict__ syn, const float *__restrict__ obs, long long n,
                               double *misfit)
{
    double acc = 0.0;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n;
         e += (long long)gridDim.x * blockDim.x) {
        const float r = syn[e] - obs[e];
        syn[e] = r;
        acc += (double)r * (double)r;
    }
    if (misfit != nullptr) block_sum_add(0.5 * acc, misfit); // uniform over the grid
}

// Time-integral misfit of Eq. 2 on residual traces r[s][n][rec] (in place):
// y^n = dt sum_{k<=n} r^k (inclusive rectangle rule), misfit += 1/2 sum y^2,
// then the adjoint source a^n = dt sum_{k>=n} y^k = (C^T C r)^n overwrites r.
// One thread per trace; compensated (Kahan) FP32 sums along time.
__global__ void k_time_integral(float *__restrict__ r, int ns, int nt, int nrec, float dt,
                                double *misfit)
{
    const long long tr = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    double acc = 0.0;
    if (tr < (long long)ns * nrec) {
        const int s = (int)(tr / nrec), q = (int)(tr - (long long)s * nrec);
        float *base = r + (long long)s * nt * nrec + q;
        float sum = 0.f, cmp = 0.f;
        for (int n = 0; n < nt; ++n) {
            const float x = base[(long long)n * nrec];
            const float y = x - cmp;
            const float t = sum + y;
            cmp = (t - sum) - y;
            sum = t;
            const float yi = dt * sum;
            base[(long long)n * nrec] = yi;
            acc += (double)yi * (double)yi;
        }
        sum = 0.f;
        cmp = 0.f;
        for (int n = nt - 1; n >= 0; --n) {
            const float x = base[(long long)n * nrec];
            const float y = x - cmp;
            const float t = sum + y;
            cmp = (t - sum) - y;
            sum = t;
            base[(long long)n * nrec] = dt * sum;
        }
    }
    block_sum_add(0.5 * acc, misfit);
}

// grad(iz, ix) = 2 / (v dx^2) * sum over groups and over the padded cells
// that replicate model cell (iz, ix) of the imaging sum G.
__global__ void k_fold_grad(const Lay2D L, const float *__restrict__ acc, int groups,
                            const float *__restrict__ v, float *__restrict__ grad)
{
    const long long n = (long long)L.nz * L.nx;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n;
         e += (long long)gridDim.x * blockDim.x) {
        const int iz = (int)(e / L.nx), ix = (int)(e - (long long)iz * L.nx);
        const int ia = iz == 0 ? 0 : iz + L.P;
        const int ib = iz == L.nz - 1 ? L.nzp - 1 : iz + L.P;
        const int ja = ix == 0 ? 0 : ix + L.P;
        const int jb = ix == L.nx - 1 ? L.nxp - 1 : ix + L.P;
        float sum = 0.f;
        for (int g = 0; g < groups; ++g) {
            const float *ag = acc + (long long)g * L.nzp * L.nxp;
            for (int i = ia; i <= ib; ++i)
                for (int j = ja; j <= jb; ++j) sum += ag[(long long)i * L.nxp + j];
        }
        grad[e] = sum * (2.0f / (v[e] * L.dx * L.dx));
    }
}

// out[plane][iz][ix] = scale * sum_g acc[g][plane][iz][ix]
__global__ void k_finish_accum(long long nphys, const float *__restrict__ acc, int groups,
                               int planes, float scale, const float *__restrict__ v6, float *__restrict__ out)
{
    const long long n = nphys * planes;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n;
         e += (long long)gridDim.x * blockDim.x) {
        float sum = 0.f;
        for (int g = 0; g < groups; ++g) sum += acc[(long long)g * n + e];
        float sc = scale;
        if (v6 != nullptr) {
            // H_a's diagonal prefactor 4 / v^6 at the cell
            const float v = v6[e % nphys], v3 = v * v * v;
            sc = sc * __fdiv_rn(4.0f, v3 * v3);
        }
        out[e] = sum * sc;
    }
}

__device__ __forceinline__ float precond_scale(const float *__restrict__ sc, long long e,
                                               long long nphys, int kind, int hmax)
{
    if (kind == 1) return sc[e];
    float p = fabsf(sc[e]);
    for (int h = 1; h <= hmax; ++h) p += 2.0f * fabsf(sc[h * nphys + e]);
    return p;
}

// max over the model of the preconditioner (non-negative: float bits order
// like unsigned integers)
__global__ void k_precond_max(long long nphys, const float *__restrict__ sc, int kind, int hmax,
                              unsigned *pmax)
{
    float mx = 0.f;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < nphys;
         e += (long long)gridDim.x * blockDim.x)
        mx = fmaxf(mx, precond_scale(sc, e, nphys, kind, hmax));
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    if ((threadIdx.x & 31) == 0) atomicMax(pmax, __float_as_uint(mx));
}

__global__ void k_precond_apply(long long nphys, const float *__restrict__ g,
                                const float *__restrict__ sc, int kind, int hmax, float eps,
                                const unsigned *pmax, float *__restrict__ out)
{
    const float w = eps * __uint_as_float(*pmax);
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < nphys;
         e += (long long)gridDim.x * blockDim.x)
        out[e] = g[e] / (precond_scale(sc, e, nphys, kind, hmax) + w);
}

__global__ void k_check_finite(const float *__restrict__ x, long long n, int *status)
{
    int bad = 0;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n;
         e += (long long)gridDim.x * blockDim.x)
        if (!isfinite(x[e])) bad = 1;
    if (__any_sync(0xffffffffu, bad) && (threadIdx.x & 31) == 0) atomicOr(status, ST_NONFINITE);
}

// adj_t[m][e] = adj[shot(e)][m][rec(e)]: the adjoint source in the order of
// the backward receiver table
__global__ void k_permute_adj(const float *__restrict__ adj, const int2 *__restrict__ ent,
                              const int *__restrict__ eshot, int nent, int nt, int nrec,
                              float *__restrict__ adj_t)
{
    const long long n = (long long)nent * nt;
    for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < n;
         q += (long long)gridDim.x * blockDim.x) {
        const int m = (int)(q / nent), e = (int)(q - (long long)m * nent);
        adj_t[q] = adj[((long long)eshot[e] * nt + m) * nrec + ent[e].y];
    }
}

// ------------------------------------------------------------- snapshots
// A snapshot of the state (u^n, u^{n-1}) in 16 bits keeps u^n and the
// increment u^n - u^{n-1} separately, each scaled by its own max-abs so that
// the largest value maps to SNAP_TARGET: the increment is small compared with
// u, and rounding u^{n-1} on its own would swamp it.
constexpr float SNAP_TARGET = 16384.0f;

__device__ __forceinline__ float snap_scale(float mx) { return mx > 0.f ? SNAP_TARGET / mx : 1.0f; }

// maxes[0][s] = max |u|, maxes[1][s] = max |u - up| over shot s's field
__global__ void k_snap_absmax(const float *__restrict__ u, const float *__restrict__ up, long long fstride,
                              float *maxes, int ns)
{
    const int s = blockIdx.y;
    const float *us = u + (long long)s * fstride, *ps = up + (long long)s * fstride;
    float mu = 0.f, md = 0.f;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < fstride;
         e += (long long)gridDim.x * blockDim.x) {
        const float a = us[e];
        mu = fmaxf(mu, fabsf(a));
        md = fmaxf(md, fabsf(a - ps[e]));
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        mu = fmaxf(mu, __shfl_xor_sync(0xffffffffu, mu, o));
        md = fmaxf(md, __shfl_xor_sync(0xffffffffu, md, o));
    }
    if ((threadIdx.x & 31) == 0) {
        atomicMax(reinterpret_cast<unsigned *>(maxes) + s, __float_as_uint(mu));
        atomicMax(reinterpret_cast<unsigned *>(maxes) + ns + s, __float_as_uint(md));
    }
}

template <typename H>
__device__ __forceinline__ H to16(float x);
template <>
__device__ __forceinline__ __nv_bfloat16 to16<__nv_bfloat16>(float x) { return __float2bfloat16_rn(x); }
template <>
__device__ __forceinline__ __half to16<__half>(float x) { return __float2half_rn(x); }
__device__ __forceinline__ float from16(__nv_bfloat16 x) { return __bfloat162float(x); }
__device__ __forceinline__ float from16(__half x) { return __half2float(x); }

// dst [2][ns][fstride]: u * s_u, (u - up) * s_d
template <typename H>
__global__ void k_snap_encode(const float *__restrict__ u, const float *__restrict__ up, int ns, long long fstride,
                              const float *__restrict__ maxes, H *__restrict__ dst)
{
    const long long n = (long long)ns * fstride;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n;
         e += (long long)gridDim.x * blockDim.x) {
        const int s = (int)(e / fstride);
        const float a = u[e];
        dst[e] = to16<H>(a * snap_scale(maxes[s]));
        dst[n + e] = to16<H>((a - up[e]) * snap_scale(maxes[ns + s]));
    }
}

// u = a / s_u, up = u - d / s_d
template <typename H>
__global__ void k_snap_decode(const H *__restrict__ src, const float *__restrict__ maxes, int ns, long long fstride,
                              float *__restrict__ u, float *__restrict__ up)
{
    const long long n = (long long)ns * fstride;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n;
         e += (long long)gridDim.x * blockDim.x) {
        const int s = (int)(e / fstride);
        const float a = from16(src[e]) / snap_scale(maxes[s]);
        u[e] = a;
        up[e] = a - from16(src[n + e]) / snap_scale(maxes[ns + s]);
    }
}

int grid_for(long long n)
{
    long long b = (n + NT1 - 1) / NT1;
    if (b < 1) b = 1;
    if (b > 152 * 16) b = 152 * 16;
    return (int)b;
}

} // namespace

cudaError_t launch_prep_c2(const Lay2D &L, const float *v, float *c2, float *damp, float cfl_limit,
                           int *status, cudaStream_t st)
{
    k_prep_c2<<<grid_for((long long)L.nzp * L.nxp), NT1, 0, st>>>(L, v, c2, damp, cfl_limit, status);
    return cudaGetLastError();
}

cudaError_t launch_prep_dc2(const Lay2D &L, const float *v, const float *dv, const float *c2, float *dc2,
                            cudaStream_t st)
{
    k_prep_dc2<<<grid_for((long long)L.nzp * L.nxp), NT1, 0, st>>>(L, v, dv, c2, dc2);
    return cudaGetLastError();
}

cudaError_t launch_prep_dext(const Lay2D &L, const float *v, const float *dv_ext, const float *c2, int hext, int he,
                             float *dext, cudaStream_t st)
{
    k_prep_dext<<<grid_for((long long)L.nzp * L.nxp * (2 * he + 1)), NT1, 0, st>>>(L, v, dv_ext, c2, hext, he, dext);
    return cudaGetLastError();
}

cudaError_t launch_fold_ext(const Lay2D &L, const float *acc, int he, int hext, const float *v, float *image,
                            cudaStream_t st)
{
    k_fold_ext<<<grid_for((long long)L.nz * L.nx * (2 * hext + 1)), NT1, 0, st>>>(L, acc, he, hext, v, image);
    return cudaGetLastError();
}

cudaError_t launch_pm_factor(int nz, int nx, float dx, float xmin, float xmax, float zr, float *out,
                             cudaStream_t st)
{
    k_pm_factor<<<grid_for((long long)nz * nx), NT1, 0, st>>>(nz, nx, dx, xmin, xmax, zr, out);
    return cudaGetLastError();
}

cudaError_t launch_pm_accumulate(int nz, int nx, float dx, float xmin, float xmax, float zr, const float *illum,
                                 float *out, cudaStream_t st)
{
    k_pm_accumulate<<<grid_for((long long)nz * nx), NT1, 0, st>>>(nz, nx, dx, xmin, xmax, zr, illum, out);
    return cudaGetLastError();
}

cudaError_t launch_wait_selftest(uint64_t limit_ns, int *status, cudaStream_t st)
{
    k_wait_selftest<<<1, 32, 0, st>>>(limit_ns, status);
    return cudaGetLastError();
}

cudaError_t launch_replicate_row(const float *src, int n, int rows, float *dst, cudaStream_t st)
{
    k_replicate_row<<<grid_for((long long)n * rows), NT1, 0, st>>>(src, n, rows, dst);
    return cudaGetLastError();
}

cudaError_t launch_scale_product(long long nphys, int planes, const float *scale, const float *recv, int rn,
                                 float *out, cudaStream_t st)
{
    k_scale_product<<<grid_for(nphys * planes), NT1, 0, st>>>(nphys, planes, scale, recv, rn, out);
    return cudaGetLastError();
}

cudaError_t launch_prep3d(const Lay3D &L, const float *v, float *c2, float *damp, float cfl_limit, int *status,
                          cudaStream_t st)
{
    k_prep3d<<<grid_for((long long)L.nzp * L.nyp * L.nxp), NT1, 0, st>>>(L, v, c2, damp, cfl_limit, status);
    return cudaGetLastError();
}

cudaError_t launch_fold_grad3d(const Lay3D &L, const float *acc, const float *v, float *grad, cudaStream_t st)
{
    k_fold_grad3d<<<grid_for((long long)L.nz * L.ny * L.nx), NT1, 0, st>>>(L, acc, v, grad);
    return cudaGetLastError();
}

cudaError_t launch_residual_ols(float *syn, const float *obs, long long n, double *misfit,
                                cudaStream_t st)
{
    k_residual_ols<<<grid_for(n / 4 + 1), NT1, 0, st>>>(syn, obs, n, misfit);
    return cudaGetLastError();
}

cudaError_t launch_time_integral(float *r, int ns, int nt, int nrec, float dt, double *misfit,
                                 cudaStream_t st)
{
    const long long ntr = (long long)ns * nrec;
    const int blocks = (int)((ntr + NT1 - 1) / NT1);
    if (blocks > 0) k_time_integral<<<blocks, NT1, 0, st>>>(r, ns, nt, nrec, dt, misfit);
    return cudaGetLastError();
}

cudaError_t launch_fold_grad(const Lay2D &L, const float *acc, int groups, const float *v,
                             float *grad, cudaStream_t st)
{
    k_fold_grad<<<grid_for((long long)L.nz * L.nx), NT1, 0, st>>>(L, acc, groups, v, grad);
    return cudaGetLastError();
}

cudaError_t launch_finish_accum_n(long long nphys, const float *acc, int groups, int planes, float scale,
                                  float *out, cudaStream_t st, const float *v6)
{
    k_finish_accum<<<grid_for(nphys * planes), NT1, 0, st>>>(nphys, acc, groups, planes, scale, v6, out);
    return cudaGetLastError();
}

cudaError_t launch_finish_accum(const Lay2D &L, const float *acc, int groups, int planes,
                                float scale, float *out, cudaStream_t st, const float *v6)
{
    return launch_finish_accum_n((long long)L.nz * L.nx, acc, groups, planes, scale, out, st, v6);
}

cudaError_t launch_precond(const Lay2D &L, const float *grad, const float *scale, int kind,
                           int hmax, float eps, float *out, unsigned *pmax, cudaStream_t st)
{
    return launch_precond_n((long long)L.nz * L.nx, grad, scale, kind, hmax, eps, out, pmax, st);
}

cudaError_t launch_precond_n(long long nphys, const float *grad, const float *scale, int kind, int hmax, float eps,
                             float *out, unsigned *pmax, cudaStream_t st)
{
    cudaError_t e = cudaMemsetAsync(pmax, 0, sizeof(unsigned), st);
    if (e != cudaSuccess) return e;
    k_precond_max<<<grid_for(nphys), NT1, 0, st>>>(nphys, scale, kind, hmax, pmax);
    k_precond_apply<<<grid_for(nphys), NT1, 0, st>>>(nphys, grad, scale, kind, hmax, eps, pmax, out);
    return cudaGetLastError();
}

cudaError_t launch_snap_absmax(const float *u, const float *up, int ns, long long fstride, float *maxes,
                               cudaStream_t st)
{
    cudaError_t e = cudaMemsetAsync(maxes, 0, 2 * (size_t)ns * sizeof(float), st);
    if (e != cudaSuccess) return e;
    int bx = (int)((fstride / 4 + NT1 - 1) / NT1);
    if (bx > 64) bx = 64;
    if (bx < 1) bx = 1;
    k_snap_absmax<<<dim3(bx, ns), NT1, 0, st>>>(u, up, fstride, maxes, ns);
    return cudaGetLastError();
}

cudaError_t launch_snap_encode(const float *u, const float *up, int ns, long long fstride, const float *maxes,
                               int prec, void *dst, cudaStream_t st)
{
    const long long n = (long long)ns * fstride;
    if (prec == 1)
        k_snap_encode<__nv_bfloat16><<<grid_for(n / 4 + 1), NT1, 0, st>>>(u, up, ns, fstride, maxes,
                                                                          static_cast<__nv_bfloat16 *>(dst));
    else
        k_snap_encode<__half><<<grid_for(n / 4 + 1), NT1, 0, st>>>(u, up, ns, fstride, maxes, static_cast<__half *>(dst));
    return cudaGetLastError();
}

cudaError_t launch_snap_decode(const void *src, const float *maxes, int prec, int ns, long long fstride, float *u,
                               float *up, cudaStream_t st)
{
    const long long n = (long long)ns * fstride;
    if (prec == 1)
        k_snap_decode<__nv_bfloat16><<<grid_for(n / 4 + 1), NT1, 0, st>>>(static_cast<const __nv_bfloat16 *>(src),
                                                                          maxes, ns, fstride, u, up);
    else
        k_snap_decode<__half><<<grid_for(n / 4 + 1), NT1, 0, st>>>(static_cast<const __half *>(src), maxes, ns,
                                                                   fstride, u, up);
    return cudaGetLastError();
}

cudaError_t launch_permute_adj(const float *adj, const int2 *ent, const int *eshot, int nent, int nt, int nrec,
                               float *adj_t, cudaStream_t st)
{
    k_permute_adj<<<grid_for((long long)nent * nt / 4 + 1), NT1, 0, st>>>(adj, ent, eshot, nent, nt, nrec, adj_t);
    return cudaGetLastError();
}

cudaError_t launch_check_finite(const float *x, long long n, int *status, cudaStream_t st)
{
    k_check_finite<<<grid_for(n), NT1, 0, st>>>(x, n, status);
    return cudaGetLastError();
}

} // namespace fwi
