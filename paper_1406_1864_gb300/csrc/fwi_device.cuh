// fwi_device.cuh -- device helpers shared by the 2-D and 3-D step kernels:
// the 8th-order weights and the second-difference Laplacian on FP32 lane
// pairs, and the PTX wrappers (mbarrier, TMA) with bounded waits.
#pragma once

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

// Lhat u in second-difference form: q = sum_k W_k ((x_{-k} + x_{+k} - 2c) +
// (z_{-k} + z_{+k} - 2c)), smallest weights first. The differences vanish
// exactly for a constant field and keep the rounding of q relative to the
// field's curvature rather than to its value. The forward and backward
// kernels both evaluate it with lap8x2 below, so q is bitwise the same in
// both passes.

// ---- paired FP32 (two lanes per instruction; each lane rounds exactly like
// the scalar operation, so paired and scalar code give identical bits)
__device__ __forceinline__ float2 f2(float a, float b) { return make_float2(a, b); }
__device__ __forceinline__ float2 add2(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 mul2(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float2 fma2(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
// a - b, one rounding
__device__ __forceinline__ float2 sub2(float2 a, float2 b) { return __ffma2_rn(b, make_float2(-1.f, -1.f), a); }
__device__ __forceinline__ float2 lo2(const float4 &v) { return make_float2(v.x, v.y); }
__device__ __forceinline__ float2 hi2(const float4 &v) { return make_float2(v.z, v.w); }
__device__ __forceinline__ float2 half2of(const float4 &v, int h) { return h == 0 ? lo2(v) : hi2(v); }

// Lhat for two adjacent points: xs[k-1], zs[k-1] are the neighbour pair sums
// at distance k along x and z.
__device__ __forceinline__ float2 lap8x2(float2 c, const float2 (&xs)[4], const float2 (&zs)[4])
{
    const float2 m2 = make_float2(-2.f, -2.f);
    float2 q = mul2(make_float2(W4, W4), add2(fma2(c, m2, xs[3]), fma2(c, m2, zs[3])));
    q = fma2(make_float2(W3, W3), add2(fma2(c, m2, xs[2]), fma2(c, m2, zs[2])), q);
    q = fma2(make_float2(W2, W2), add2(fma2(c, m2, xs[1]), fma2(c, m2, zs[1])), q);
    q = fma2(make_float2(W1, W1), add2(fma2(c, m2, xs[0]), fma2(c, m2, zs[0])), q);
    return q;
}

// Lhat of the 4 points of one thread row r: x-window w (the row, w[WL] the
// first point) and the column window zc (rows r .. r+8 of the stage tile).
// ODD_SCALAR: odd-distance x pairs as two scalar adds instead of one paired
// add on moved registers (the same bits either way; the choice that the
// register allocation of each kernel prefers).
template <int WL, int NZ, bool ODD_SCALAR = true>
__device__ __forceinline__ void lap4(float2 (&q)[2], const float *w, const float4 (&zc)[NZ], int r)
{
#pragma unroll
    for (int h = 0; h < 2; ++h) {
        const int p = 2 * h;
        float2 xs[4], zs[4];
#pragma unroll
        for (int k = 1; k <= 4; ++k) {
            // even k: both pairs are aligned register pairs (one FADD2);
            // odd k: two scalar adds
            if ((k & 1) == 0 || !ODD_SCALAR)
                xs[k - 1] = add2(f2(w[WL + p - k], w[WL + p + 1 - k]), f2(w[WL + p + k], w[WL + p + 1 + k]));
            else
                xs[k - 1] = f2(w[WL + p - k] + w[WL + p + k], w[WL + p + 1 - k] + w[WL + p + 1 + k]);
            zs[k - 1] = add2(half2of(zc[r + 4 - k], h), half2of(zc[r + 4 + k], h));
        }
        q[h] = lap8x2(f2(w[WL + p], w[WL + p + 1]), xs, zs);
    }
}

// One damped leapfrog step in increment form:
//   u^{n+1} = u^n + ((1 - eta dt)(u^n - u^{n-1}) + c2 q) / (1 + eta dt),
// algebraically the update of the header; carrying the small increment
// u^n - u^{n-1} keeps the FP32 rounding at the increment's scale. Written out
// in the kernels as u + fma(c2 ia, q, kb (u - u_prev)) with ia = 1/(1 + eta dt)
// (precomputed per cell) and kb = (1 - eta dt) ia = 2 ia - 1 (exact in FP32
// for ia in (1/2, 1]); where eta = 0 it is exactly u + fma(c2, q, u - u_prev).

// The reverse step in the model (eta = 0), u^{n-1} = u^n - ((u^{n+1} - u^n)
// - c2 q^n), is written out on lane pairs in the backward kernel.

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

// p[0..3] += (a, b, c, d) as one vector reduction in L2: a warp's 32 rows of
// 4 consecutive floats touch 16 sectors instead of 64 for four scalar
// reductions. p must be 16-byte aligned.
__device__ __forceinline__ void red_add4(float *p, float a, float b, float c, float d)
{
    asm volatile("red.global.add.v4.f32 [%0], {%1, %2, %3, %4};" ::"l"(p), "f"(a), "f"(b), "f"(c), "f"(d)
                 : "memory");
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
    const uint32_t bar = smem_u32(&bars[k % STAGES]), parity = (k / STAGES) & 1;
    if (mbar_try_wait(bar, parity)) return true;
    if (mbar_wait(bar, parity, WAIT_NS)) return true;
    *s_abort = 1;
    return false;
}

constexpr int DESC_RING = 8; // item descriptors staged ahead (ring size)

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
} // namespace fwi
