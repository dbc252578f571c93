// fwi_args.h -- layouts, kernel argument blocks, tilings and status bits of
// libfwi's step kernels (CUDA, sm_103a): the data the kernels are compiled
// against. Launchers and host helpers are declared in fwi_internal.h. Not
// part of the public ABI.
#pragma once

#include <cstddef>
#include <cstdint>
#include <cuda.h>
#include <cuda_runtime.h>

#include "fwi.h"

namespace fwi {

// ---------------------------------------------------------------- layout
// A padded 2-D field (model + sponge, nzp x nxp) is stored row-major with a
// zero ghost frame so that stencil and offset reads never leave the buffer:
// GZ rows above and below, GXL columns on the left (128-byte aligned start of
// the padded row) and at least GXR columns on the right. Ghost cells are set
// to zero once per call and never written.
constexpr int GZ = 4;
constexpr int GXL = 32;
constexpr int GXR = 16;
constexpr int RADIUS = 4;          // half-width of the 8th-order stencil
constexpr int HMAX_LIMIT = 12;     // largest offset of the offset Hessian

// Tile of the 2-D step kernels: TX columns (16 threads x float4) by
// TZ = 8 * RZ rows (8 thread rows x RZ rows each), 128 threads.
constexpr int TX = 64;
constexpr int TPB = 128;

struct Lay2D {
    int nz, nx, P;        // model and sponge
    int nzp, nxp;         // padded grid
    int pitch;            // floats per stored row
    int rows;             // stored rows = nzp + 2 GZ
    long long fstride;    // floats per stored field (rows * pitch), 64-float aligned
    int nband;            // sponge cells of one field (checkpointed each step)
    int nbandp;           // per-step checkpoint stride: nband rounded up to 4 floats
    float dt, dx;
    float etamax_dt;      // eta_max * dt
    float inv_p2;         // 1 / P^2
};

__host__ __device__ inline long long fidx(const Lay2D &L, int i, int j)
{
    return (long long)(i + GZ) * L.pitch + (j + GXL);
}

// cells into the sponge along one axis (0 inside the model)
__host__ __device__ inline int sponge_depth(int i, int P, int n)
{
    return i < P ? P - i : (i >= P + n ? i - (P + n - 1) : 0);
}

// index of sponge cell (i, j) in the per-step checkpoint of one field;
// -1 for model cells. Order: top P rows, then (left P, right P) per model row,
// then bottom P rows.
__host__ __device__ inline int band_index(const Lay2D &L, int i, int j)
{
    const int P = L.P;
    if (i < P) return i * L.nxp + j;
    if (i >= P + L.nz) return P * L.nxp + 2 * P * L.nz + (i - P - L.nz) * L.nxp + j;
    if (j < P) return P * L.nxp + (i - P) * 2 * P + j;
    if (j >= P + L.nx) return P * L.nxp + (i - P) * 2 * P + P + (j - P - L.nx);
    return -1;
}

// ------------------------------------------------------- receiver tables
// Receivers of each (tile, shot), for a tiling of TX x TZ: entries
// [ptr[t*ns+s], ptr[t*ns+s+1]) of ent, each {local = zl*TX + xl, r}.
struct RecTable {
    const int *ptr;
    const int2 *ent;
};

// ------------------------------------------------------------ kernel args
struct StepCommon {
    Lay2D L;
    const float *c2;       // (v dt / dx)^2, field layout
    const float *damp;     // 1 / (1 + eta dt), field layout (1 in the model)
    const int *src_off;    // [ns] field offset of each source cell
    const int2 *src_ij;    // [ns] padded (row, column) of each source cell
    const float *wav;      // [ns][nt]
    float src_scale;       // dx^(2 - ndim)
    int ns, nt, nrec;
    int ntx, ntz;          // tiles of this launch's tiling
    int *status;           // device status flags
    int *sched;            // this launch's chunk counter (zero at launch)
    int chunk;             // shots per chunk of the work schedule
};

// Time-loop kernels read their tiles with TMA: 3-D tensor maps over the
// [ns][rows][pitch] wavefield buffers, one "halo" box (tile + stencil halo)
// and one "point" box (tile only) per buffer. CUtensorMap carries its own
// alignment and is read from the kernel's parameter space (__grid_constant__).
struct FwdArgs {
    CUtensorMap tm_cur;    // u^n, halo box
    CUtensorMap tm_prev;   // u^{n-1}, point box
    StepCommon c;
    const float *uin;      // u^n (the buffer of tm_cur): the offset-Hessian sums of the
                           // split variants read it
    float *uout;           // u^{n+1} is written here (the u^{n-1} buffer, or a
                           // segment slot when re-propagating from a snapshot)
    float *qout;           // re-propagation: q^n = Lhat u^n + f delta_s (in place of
                           // u^{n-1}) for the backward step's imaging, else null
    float *band;           // [ns][nt][nbandp] checkpoints (u^{n+1} stored) or null
    float *seis;           // [ns][nt][nrec] traces or null
    float *acc_illum;      // [nz][nx] or null (red.add)
    float *acc_offh;       // [hmax+1][nz][nx] or null (red.add)
    RecTable rt;
    int n;                 // time level of u^n
    int last;              // n == nt-1: extract and accumulate only
    int illum_utt;         // accumulate (u^{n+1}-2u^n+u^{n-1})^2 instead of u^2
    int hmax;
};

struct BwdArgs {
    CUtensorMap tm_ub;     // u^{m-1}, halo box (qin: q^{m-1}, point box)
    CUtensorMap tm_pa;     // psi^{m+1}, halo box
    CUtensorMap tm_ua;     // u^m, point box
    CUtensorMap tm_pb;     // psi^{m+2}, point box
    StepCommon c;
    float *ua;             // u^m buffer: u^{m-2} is written here
    float *pb;             // psi^{m+2} buffer: psi^m is written here
    const float *band;     // [ns][nt][nbandp] checkpoints
    const float *adj;      // [nt][nent] adjoint source in receiver-table order, or null
    int nent;              // ns * nrec
    float *acc_grad;       // [nzp][nxp] sum psi^m * (Lhat u^{m-1} + f delta_s) (red.add)
    float *acc_ext;        // extended imaging: [2 HE + 1][nzp][nxp] sums psi^m(y) q^{m-1}(y + 2h)
                           // at (h + HE, y) (red.add), or null
    RecTable rt;
    float adj_scale;       // dx^2
    int m;
    int recon;             // 1: rebuild u^{m-2} (model) / restore it (sponge);
                           // 0: u^{m-1} comes from a re-propagated segment
    int qin;               // 1: the imaging factor q^{m-1} = Lhat u^{m-1} + f delta_s
                           // is read (tm_ub), kept by the segment's re-propagation
};

// The work of one step launch: the (tile, shot) pairs of one model, or of up
// to BATCH_MAX independent models of different sizes (one argument block
// each). Chunks of the models are numbered consecutively; chunk_end[m] is the
// end of model m's. All models of a launch share the time level, the status
// flags, the chunk counter and the chunk size.
constexpr int BATCH_MAX = FWI_BATCH_MAX;
template <class A, int N>
struct Batch {
    static constexpr int NM = N;
    A m[N];
    int chunk_end[N];
    int nm;
    int chunk;  // shots per chunk
    int *sched; // the launch's chunk counter (zero at launch)
};

// Born (tangent-linear) step: u and du = J dv advanced together
struct BornArgs {
    CUtensorMap tm_u;      // u^n, halo box
    CUtensorMap tm_du;     // du^n, halo box
    CUtensorMap tm_up;     // u^{n-1}, point box
    CUtensorMap tm_dup;    // du^{n-1}, point box
    StepCommon c;
    const float *dc2;      // 2 c2 dv / v, field layout
    const float *dext;     // extended Born: planes h = -HE..HE (field layout, fstride apart) of
                           // D~(y, h) = 2 c2 dv(y + h, h) / v at y + h, or null
    float *uout, *duout;   // u^{n+1} and du^{n+1} written here
    float *band;           // sponge checkpoint of u^{n+1} (for an adjoint pass) or null
    float *dseis;          // [ns][nt][nrec] Born traces du^n at the receivers, or null
    RecTable rt;
    int n, last;
};

// status bits written by kernels
enum : int {
    ST_NONFINITE = 1,
    ST_BAD_VELOCITY = 2,
    ST_CFL = 4,
    ST_TIMEOUT = 8
};

// ------------------------------------------------------------- launchers
// Step kernels: `ctas` CTAs (one per resident slot) take chunks of `chunk`
// shots of one tile from an atomic counter.
struct Tiling {
    int variant;   // compiled tile variant of the kind (0 = default)
    int spi;       // shots per item (the depth of the step's tensor-map boxes)
    int tz;        // tile height
    int ntx, ntz;  // tiles
    int ctas;      // CTAs of one launch
    int chunk;     // shots per chunk
};
enum StepKind { STEP_FWD = 0, STEP_FWD_OFFH = 1, STEP_BWD = 2 };

// compiled offset counts of the extended operators go up to HEXT_MAX
constexpr int HEXT_MAX = 6;

} // namespace fwi
