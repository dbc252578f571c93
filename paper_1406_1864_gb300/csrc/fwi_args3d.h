// fwi_args3d.h -- argument blocks of the 3-D step kernels (host and device),
// kept apart from the 2-D ones in fwi_args.h.
#pragma once

#include "fwi_args.h"

namespace fwi {

// ------------------------------------------------------------------- 3-D
// Padded 3-D field [planes][rows][pitch]: z planes (GZ ghost planes above and
// below), y rows (GY ghost rows on both sides), x as in 2-D (GXL / GXR ghost
// columns, pitch a multiple of 32 floats). Shots are stacked by fstride.
constexpr int GY = 4;
constexpr int TY3 = 8; // 3-D tiles: 64 (x) x 8 (y) columns, marched along z

struct Lay3D {
    int nz, ny, nx, P;
    int nzp, nyp, nxp;
    int pitch, rows, planes; // floats per row, rows per plane, planes per field
    long long plane;         // floats per plane
    long long fstride;       // floats per field (aligned)
    float dt, dx;
    float etamax_dt, inv_p2;
};

__host__ __device__ inline long long fidx3(const Lay3D &L, int i, int k, int j)
{
    return (long long)(i + GZ) * L.plane + (long long)(k + GY) * L.pitch + GXL + j;
}

struct Step3Common {
    Lay3D L;
    const float *c2;    // (v dt / dx)^2, field layout
    const float *damp;  // 1 / (1 + eta dt), field layout
    const int4 *src;    // [ns] padded (z, y, x) of each source
    const float *wav;   // [ns][nt]
    float src_scale;    // dx^(2 - ndim) = 1/dx
    int ns, nt, nrec;
    int nty, ntx;       // tiles along y and x
    int nseg, segl;     // z-segments of a column and their length in planes
    int *status;        // device status flags
    int *sched;         // this launch's item counter (zero at launch)
};

// receivers of each (tile, shot): ptr[tile * ns + s] .. ptr[... + 1] into ent
// = (padded plane, y * 64 + x within the tile, receiver, 0), sorted by plane;
// zr[tile * ns + s] = (first, last) plane with receivers (last < first: none)
struct Rec3Table {
    const int *ptr;
    const int4 *ent;
    const int2 *zr;
};

struct Fwd3Args {
    CUtensorMap tm_u;    // u^n, halo box (TX+8) x (TY3+8) of one plane
    CUtensorMap tm_upt;  // u^n, point box TX x TY3
    CUtensorMap tm_prev; // u^{n-1}, point box
    CUtensorMap tm_c2;   // c2, point box (one field)
    CUtensorMap tm_damp; // damping factor, point box (one field)
    Step3Common c;
    const float *uin;    // u^n (the buffer of tm_u / tm_upt): a segment's first planes
    float *uout;         // u^{n+1} written here (null: not written)
    float *qout;         // null, or q^n = Lhat u^n + f delta_s / dx written here; may be the
                         // u^{n-1} buffer (each point's u^{n-1} is read before its q^n is written)
    float *seis;         // [ns][nt][nrec] or null
    float *acc_illum;    // [nz][ny][nx] or null (red.add)
    Rec3Table rt;
    int n, last, illum_utt;
};

struct Bwd3Args {
    CUtensorMap tm_q;         // q^{m-1} = Lhat u^{m-1} + f delta_s / dx (kept by the re-propagation): point box
    CUtensorMap tm_p, tm_ppt; // psi^{m+1}: halo, point boxes
    CUtensorMap tm_pb;        // psi^{m+2}: point box
    CUtensorMap tm_c2, tm_damp;
    Step3Common c;
    const float *pin;         // psi^{m+1} (the buffer of tm_p): a segment's first planes
    float *pb;                // psi^m written here (the psi^{m+2} buffer)
    const float *adj;         // [ns][nt][nrec] adjoint source or null
    float *acc_grad;          // [nzp][nyp][nxp] (red.add)
    Rec3Table rt;
    float adj_scale;          // dx^2
    int m;
};

struct Tiling3 {
    int nty, ntx, ctas;
    int nseg, segl; // z-segments per column (items: segment x tile x shot), planes per segment
};

} // namespace fwi
