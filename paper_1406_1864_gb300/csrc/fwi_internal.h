// fwi_internal.h -- launchers and host helpers shared by the translation
// units of libfwi (CUDA, sm_103a); the layouts and kernel arguments they take
// are in fwi_args.h. Not part of the public ABI.
#pragma once

#include "fwi_args.h"
#include "fwi_args3d.h"

namespace fwi {
// 3-D steps: compiled variants of the forward (backward = false) or backward
// step, the autotuned one of a problem shape (0 if none is kept), the
// tiling of a variant (an out-of-range one is taken as 0), launches
int step3_variants(bool backward);
int step3_variant_for(const Lay3D &L, int ns, bool backward);
int step3_segments_for(const Lay3D &L, int ns, bool backward); // 0: chosen per launch shape
void step3_tuned_store(const Lay3D &L, int ns, bool backward, int variant, int nseg);
void step3_tuned_clear();
// nseg: z-segments per column, 0 to choose them from the items and resident CTAs
Tiling3 make_tiling3(const Lay3D &L, int ns, bool backward, int variant, int nseg = 0);
// tensor map over nfields 3-D fields with a box of bx x by cells of one plane
bool encode_field_map3(CUtensorMap *map, const float *base, const Lay3D &L, int nfields, int bx, int by);
cudaError_t launch_fwd3d(const Fwd3Args &a, const Tiling3 &t, int variant, cudaStream_t st);
cudaError_t launch_bwd3d(const Bwd3Args &a, const Tiling3 &t, int variant, cudaStream_t st);
// offset-Hessian sums of up to two 3-D levels (u0, u1; null: skipped):
// acc[h][x] += sum_levels sum_s u_s(x + h e_x) u_s(x - h e_x), h <= hmax
cudaError_t launch_offh3d(const float *u0, const float *u1, const Lay3D &L, int ns, int hmax, float *acc,
                          cudaStream_t st);
cudaError_t launch_prep3d(const Lay3D &L, const float *v, float *c2, float *damp, float cfl_limit, int *status,
                          cudaStream_t st);
cudaError_t launch_fold_grad3d(const Lay3D &L, const float *acc, const float *v, float *grad, cudaStream_t st);
// finish / precondition over nphys model cells (any dimension)
cudaError_t launch_finish_accum_n(long long nphys, const float *acc, int groups, int planes, float scale,
                                  float *out, cudaStream_t st, const float *v6 = nullptr);
cudaError_t launch_precond_n(long long nphys, const float *grad, const float *scale, int kind, int hmax, float eps,
                             float *out, unsigned *pmax, cudaStream_t st);

// tiling of a kind of step: the given variant / chunk, or (variant < 0,
// chunk <= 0) the autotuned ones of this problem shape, else the defaults
// (hmax: the offset Hessian's largest offset, for the variants of
// STEP_FWD_OFFH, which cover hmax up to a compiled count)
Tiling make_tiling(const Lay2D &L, int ns, StepKind kind, int variant = -1, int chunk = 0, int hmax = HMAX_LIMIT);
bool step_variant_valid(StepKind kind, int variant, int hmax);
// box sizes (x, y) of the halo and point tiles of a step kernel
void step_boxes(StepKind kind, const Tiling &t, int &hx, int &hy, int &px, int &py);
// most tiles of any variant (receiver tables are sized for it)
int max_tiles(const Lay2D &L);
// autotuning: compiled variants and chunk sizes of a kind, and the choices
// kept per (kind, padded shape, shots) for the process
int step_variants(StepKind kind);
int step_chunks(StepKind kind, const int **chunks);
void step_tuned_store(StepKind kind, const Lay2D &L, int ns, int variant, int chunk);
bool step_tuned_lookup(StepKind kind, const Lay2D &L, int ns, int &variant, int &chunk);
void step_tuned_clear();

bool encode_field_map(CUtensorMap *map, const float *base, const Lay2D &L, int nfields, int bx, int by,
                      int bz = 1);
cudaError_t launch_fwd_step(const FwdArgs &a, const Tiling &t, bool with_offh, cudaStream_t st);
// with the offset Hessian: does the tiling's variant launch k_offh_level after the plain step
bool fwd_split(const Tiling &t, bool with_offh);
cudaError_t launch_bwd_step(const BwdArgs &a, const Tiling &t, cudaStream_t st);
// one launch over the (tile, shot) pairs of nm <= BATCH_MAX models at the
// same time level (per-model arguments and tilings of the same kind)
cudaError_t launch_fwd_batch(const FwdArgs *a, const Tiling *t, int nm, bool with_offh, cudaStream_t st);
cudaError_t launch_bwd_batch(const BwdArgs *a, const Tiling *t, int nm, cudaStream_t st);
// Born step over all shots (the backward step's tiling: two halo fields)
cudaError_t launch_born_step(const BornArgs &a, const Tiling &t, cudaStream_t st);
// extended operators (Eq. 5, Eq. 6), offsets h = -he..he, he in {2, 4, 6};
// tiles of 64 x 8 (t.tz == 8); the halo boxes are TX + 2 (RADIUS + 2 he) wide
int ext_kernel_he(int hext); // the compiled offset count that covers |h| <= hext
void ext_boxes(int he, const Tiling &t, int &hx, int &hy, int &px, int &py);
cudaError_t launch_bwd_ext_step(const BwdArgs &a, const Tiling &t, int he, cudaStream_t st);
cudaError_t launch_born_ext_step(const BornArgs &a, const Tiling &t, int he, cudaStream_t st);
// D~(y, h) = 2 c2(y + h) dv(y + h, h) / v(y + h) on the padded grid for |h| <= hext (edge-replicated
// dv_ext [2 hext + 1][nz][nx]), zero where y + h leaves the padded grid or |h| > hext; planes
// h = -he..he, fstride apart
cudaError_t launch_prep_dext(const Lay2D &L, const float *v, const float *dv_ext, const float *c2, int hext, int he,
                             float *dext, cudaStream_t st);
// image(x, h) = sum over the padded cells x' folding into x of 2 v(x') / (v(x' - h)^2 dx^2) acc(x' - h, h),
// |h| <= hext, image [2 hext + 1][nz][nx]; acc [2 he + 1][nzp][nxp]
cudaError_t launch_fold_ext(const Lay2D &L, const float *acc, int he, int hext, const float *v, float *image,
                            cudaStream_t st);
// dc2 = 2 c2 dv / v on the padded grid (edge-replicated dv)
cudaError_t launch_prep_dc2(const Lay2D &L, const float *v, const float *dv, const float *c2, float *dc2,
                            cudaStream_t st);

// auxiliary kernels (fwi_aux.cu)
// receiver factor of the diagonal Hessian and its product with a scale
cudaError_t launch_pm_factor(int nz, int nx, float dx, float xmin, float xmax, float zr, float *out,
                             cudaStream_t st);
cudaError_t launch_replicate_row(const float *src, int n, int rows, float *dst, cudaStream_t st);
// one warp waiting (bounded by limit_ns) on an mbarrier no thread arrives at
cudaError_t launch_wait_selftest(uint64_t limit_ns, int *status, cudaStream_t st);
cudaError_t launch_pm_accumulate(int nz, int nx, float dx, float xmin, float xmax, float zr, const float *illum,
                                 float *out, cudaStream_t st);
cudaError_t launch_scale_product(long long nphys, int planes, const float *scale, const float *recv, int rn,
                                 float *out, cudaStream_t st);
cudaError_t launch_prep_c2(const Lay2D &L, const float *v, float *c2, float *damp, float cfl_limit,
                           int *status, cudaStream_t st);
cudaError_t launch_residual_ols(float *syn, const float *obs, long long n, double *misfit,
                                cudaStream_t st);
cudaError_t launch_time_integral(float *r, int ns, int nt, int nrec, float dt, double *misfit,
                                 cudaStream_t st);
cudaError_t launch_fold_grad(const Lay2D &L, const float *acc, int groups, const float *v,
                             float *grad, cudaStream_t st);
// (v6: multiply by 4 / v^6 at each cell, v the physical velocity, or null)
cudaError_t launch_finish_accum(const Lay2D &L, const float *acc, int groups, int planes,
                                float scale, float *out, cudaStream_t st, const float *v6 = nullptr);
cudaError_t launch_precond(const Lay2D &L, const float *grad, const float *scale, int kind,
                           int hmax, float eps, float *out, unsigned *pmax, cudaStream_t st);
cudaError_t launch_check_finite(const float *x, long long n, int *status, cudaStream_t st);
// snapshots of (u^n, u^{n-1}) in 16 bits: u and u - u_prev, each scaled by
// its own max-abs (prec 1: bfloat16, 2: float16)
cudaError_t launch_snap_absmax(const float *u, const float *up, int ns, long long fstride, float *maxes,
                               cudaStream_t st);
cudaError_t launch_snap_encode(const float *u, const float *up, int ns, long long fstride, const float *maxes,
                               int prec, void *dst, cudaStream_t st);
cudaError_t launch_snap_decode(const void *src, const float *maxes, int prec, int ns, long long fstride, float *u,
                               float *up, cudaStream_t st);
cudaError_t launch_permute_adj(const float *adj, const int2 *ent, const int *eshot, int nent, int nt, int nrec,
                               float *adj_t, cudaStream_t st);

} // namespace fwi
