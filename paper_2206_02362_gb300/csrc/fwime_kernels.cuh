// Internal kernel interfaces of libfwime (not part of the C ABI).
//
// Field layout on the device: every wavefield of one shot is a padded grid
// [NZ][NXP] of FP32, NZ = nz + 2(W+4), NX = nx + 2(W+4), NXP = NX rounded up to
// a multiple of 32 floats (128-byte rows).  The physical point (iz, ix) sits at
// (iz + W + 4, ix + W + 4).  "Active" points are 4 <= IZ < NZ-4, 4 <= IX < NX-4;
// every other point of every field is zero and stays zero because the sponge
// factors gz[IZ] gx[IX] (and c) are zero there.
//
// Shots advanced together ("a batch") are consecutive fields P = NZ*NXP apart;
// a ring of K time slots holds [K][S][P].
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include <cmath>

namespace fwk {

constexpr int STRIP = 128;      // x-points per warp in the stencil kernel (32 lanes x float4)
constexpr int PROP_WARPS = 4;   // warps per CTA in the stencil kernel
constexpr int EXT_TX = 128;     // x-points per CTA in the scatter / imaging kernels
constexpr int MAX_NH = 201;     // largest supported number of subsurface offsets
#ifndef FWIME_EXT_STAGES
#define FWIME_EXT_STAGES 6
#endif
constexpr int EXT_STAGES = FWIME_EXT_STAGES;   // cp.async pipeline depth of the imaging kernels (even, >= 4)

// status bits latched by kernels
constexpr int ST_CFL = 1;
constexpr int ST_BADV = 2;

// Largest eigenvalue of -h^2 D2 for the 8th-order second-derivative stencil (its symbol at the Nyquist
// wavenumber: 205/72 + 2 (8/5 + 1/5 + 8/315 + 1/560)).  The leapfrog scheme is stable while
// dt v sqrt(LAMBDA_MAX (1/dx^2 + 1/dz^2)) < 2.
constexpr double LAMBDA_MAX = 6.5015873015873;

// Square of the largest velocity the scheme accepts at (dt, dx, dz), compared against v^2 by k_prep.
inline float cfl_vmax2(float dt, float dx, float dz)
{
    const double lim = 2.0 / ((double)dt * std::sqrt(LAMBDA_MAX * (1.0 / ((double)dx * dx) + 1.0 / ((double)dz * dz))));
    return (float)(lim * lim);
}

struct PropArgs {
    int NZ, NXP, zchunk, nstrip, nchunk;
    long long P;                   // floats per shot field
    float ax[5], az[5];            // 8th-order coefficients divided by dx^2, dz^2
    float inv_dt2;
    const float *c, *gz, *gx;      // model: c = v^2 dt^2 [P], sponge factors [NZ], [NXP]
    const float *cur;              // q^n           (shot s at + s*P)
    const float *prev;             // q^{n-1}
    float *out;                    // q^{n+1}       (may alias prev)
    float *d2;                     // optional (q^{n+1} - 2 q^n + q^{n-1}) / dt^2
    // optional point source: s += amp at src_off[s]
    const int *src_off;
    const float *src_amp;          // amplitude of shot s at src_amp[s * src_stride]
    long long src_stride;
    float src_scale;               // 1 / (dx dz)
    // optional dense local source: s += sum_i alpha_i f_i + coef * fc
    const float *f0, *f1, *f2;
    float a0, a1, a2;
    const float *coef, *fc;
    // rows [zs_lo, zs_hi) (the physical rows): the only rows where the local sources may be nonzero
    // (read there only, zero elsewhere) and where D2t is written (its readers, the extension and
    // imaging kernels, read physical rows only)
    int zs_lo, zs_hi;
    int naux_max;                  // rows per aux stage (set by launch_prop)
    // optional receiver recording of the INPUT field: d[s * rec_dstride + r] (=, or += with rec_acc)
    // = cur[s * P + rec_off[r]] for r < nrec, done by the first CTA of every shot (cur is complete
    // before the launch, so any CTA may read it)
    const int *rec_off;
    float *rec_d;
    long long rec_dstride;
    int nrec, rec_acc;
    // optional receiver injection into the OUTPUT field: out(rec_r) += c(rec_r) inj_val[s * inj_vstride + r]
    // (the transpose of recording, as k_points injects it).  inj_map[(z - inj_lo) * NXP + x] is the first
    // receiver at padded point (z, x) of the rows [inj_lo, inj_hi) or -1, inj_next[r] the next receiver at
    // the same point or -1.
    const int *inj_map, *inj_next;
    const float *inj_val;
    long long inj_vstride;
    int inj_lo, inj_hi;
    // each scalar twice, the operands of the packed two-lane (f32x2) arithmetic (set by prop_pairs)
    float2 kx2[5], kz2[5], axc2, inv2, a02, a12, a22;
};

// Fills the packed-operand copies of a's coefficients (host side, after they are final).
inline void prop_pairs(PropArgs &a)
{
    for (int k = 0; k < 5; ++k) {
        a.kx2[k] = make_float2(a.ax[k], a.ax[k]);
        a.kz2[k] = make_float2(a.az[k], a.az[k]);
    }
    const float axc = a.ax[0] + a.az[0];
    a.axc2 = make_float2(axc, axc);
    a.inv2 = make_float2(a.inv_dt2, a.inv_dt2);
    a.a02 = make_float2(a.a0, a.a0);
    a.a12 = make_float2(a.a1, a.a1);
    a.a22 = make_float2(a.a2, a.a2);
}

// grouped forward: one member = one shot batch on its own grid
struct GroupMember {
    PropArgs a[2];                 // even / odd steps (cur and prev swap); src_amp = wavelet base
    int cta_begin;                 // first CTA of this member in the launch
    int ctas_per_shot;
};
struct GroupRec {
    const int *rec_off;
    const float *fA, *fB;          // the member's two wavefield buffers
    float *d;                      // data [nshot][nt][nrec]
    long long P;
    int nrec, nshot, nt, rec_begin;
};

struct PointsArgs {
    int nrec;
    long long P;
    const int *rec_off;            // [nrec] linear offsets in a field
    // record: d[s*dstride + r] (= or +=) f1[s*P + off] (+ f2[s*P + off])
    const float *f1, *f2;
    float *d;
    long long dstride;
    int accumulate;
    // inject: fld[s*P + off] += c[off] * val[s*vstride + r]   (c g at a receiver; g = 1 on the
    // physical grid, where receivers live)
    float *fld;
    const float *val;
    long long vstride;
    const float *c;
};

// A ring operand of the segment kernels: slot of time step n (pair row j) is
//   mod > 0 : (n + shift) % mod        mod == 0 : j + shift
struct RingRef {
    const float *base;
    long long slot_stride;         // floats between slots (S_cap * P)
    int mod, shift;
};

struct ExtArgs {
    int NXP, nh, hm, S, npair, n0;
    long long P;
    int z_lo, z_hi, x_lo, x_hi;    // output rows/cols processed
    int sigma;                     // +1: out(y) = sum_h W(y-h,h) D(y-2h); -1: W(y+h,h) D(y+2h)
    const float *W;                // [nh][P] weights (zero off the physical grid)
    RingRef in;                    // D
    RingRef outr;                  // output ring (written through a non-const cast)
    int accumulate;
};

enum { IMG_EXT = 0, IMG_CONTRACT = 1, IMG_LOCAL = 2 };

struct ImgArgs {
    int NXP, nh, hm, S, npair, n0;
    long long P;
    int z_lo, z_hi, x_lo, x_hi;
    RingRef D;                     // source-side field  D(x - h)
    RingRef L;                     // receiver-side field L(x + h)
    RingRef M2;                    // IMG_LOCAL: second adjoint field (may be null base)
    RingRef Ds;                    // IMG_LOCAL: scattered D2t field (may be null base)
    float alpha;                   // IMG_LOCAL: weight of D * L
    const float *pt;               // IMG_CONTRACT: p~ padded [nh][P]
    float *img;                    // IMG_EXT: [nh][P]; others: [P]
    float *img_local;              // IMG_EXT, optional: [P] += the IMG_LOCAL terms (alpha D L + D M2 + Ds L)
};

// time-lag extension: one segment [n0, n1) of output steps, S shots
struct TlagArgs {
    int NXP, nh, S, lag, nt, n0, n1;
    int jc;                        // outputs of one residue class per thread and chunk (16, 20, 24, 32: tlag_jc)
    int sigma;                     // scatter: +1 reads D at n - 2 s_i, -1 (transpose) at n + 2 s_i
    long long P;
    int z_lo, z_hi, x_lo, x_hi;    // physical rows / columns
    const float *W;                // [nh][P] weights b p~ (scatter)
    RingRef D;                     // scatter input (background D2t; adjoint field for sigma = -1), slot of step m
    RingRef E;                     // scatter output, slot of n - n0 (with shift n0 and mod: a ring indexed by n)
    RingRef L;                     // image: receiver side, slot of step n
    float *img;                    // image [nh][P]
    int accumulate;
};

// launchers (return cudaGetLastError())
cudaError_t launch_prop(const PropArgs &a, int nshot, cudaStream_t st);
cudaError_t prop_occupancy(int *blocks_per_sm);
cudaError_t launch_prop_group(const GroupMember *m, int nactive, int ctas, const GroupRec *g, int nrec_threads,
                              int step, cudaStream_t st, bool record);
cudaError_t launch_points(const PointsArgs &a, int nshot, cudaStream_t st);
cudaError_t launch_scatter(const ExtArgs &a, cudaStream_t st);
cudaError_t launch_image(const ImgArgs &a, int mode, cudaStream_t st);
cudaError_t launch_tlag_scatter(const TlagArgs &a, cudaStream_t st);
cudaError_t launch_tlag_image(const TlagArgs &a, cudaStream_t st);
int tlag_jc(int K, int lag, int nh);          // chunk length (outputs of one residue class) for segments of K steps

// model preparation
struct PrepArgs {
    int nz, nx, o, NZ, NX, NXP, W;
    float dt, cfl_limit2;          // (2 / (dt sqrt(6.5016 (1/dx^2 + 1/dz^2))))^2 = vmax^2 bound
    const float *v;                // [nz][nx]
    float *c, *gz, *gx, *bpad;     // padded outputs
    int *status;
    int fs;                        // 1: free surface at the top physical row
};
cudaError_t launch_prep(const PrepArgs &a, cudaStream_t st);
cudaError_t launch_free_surface(float *q, float *d2, int nshot, long long P, int NXP, int o, cudaStream_t st);

// elementwise helpers on padded / physical grids
cudaError_t launch_embed_scale(const float *phys, const float *scale_pad, float *out_pad, int nz, int nx,
                               int o, int NXP, float alpha, cudaStream_t st);
cudaError_t launch_ext_weights(const float *pt, const float *bpad, const float *dv, const float *v, float *Wout,
                               int nh, int nz, int nx, int o, int NXP, long long P, int mode, cudaStream_t st);
cudaError_t launch_finalize(const float *acc1, const float *acc2, const float *bpad, const float *v, float *out,
                            int nplanes, int nz, int nx, int o, int NXP, long long P, int mode, int accumulate,
                            cudaStream_t st, const float *pt = nullptr, int nh = 0);
cudaError_t launch_residual(const float *pred, const float *dobs, float *r, long long n, double *partials,
                            int nblocks, cudaStream_t st);
cudaError_t launch_sum_partials(const double *partials, int n, double *out, int accumulate, double scale,
                                cudaStream_t st);
cudaError_t launch_dso(const float *pt, int nh, long long PP, double *partials, int nblocks, cudaStream_t st);
cudaError_t launch_copy_fields(float *dst, const float *src, long long n, cudaStream_t st);
// linear spline re-parametrisation: out = S in (adjoint = 0) or S* in (tmp: nz * nxs floats)
cudaError_t launch_spline(const float *zs, int nzs, const float *xs, int nxs, int nz, int nx, float dz, float dx,
                          const float *in, float *out, float *tmp, int adjoint, int accumulate, cudaStream_t st);
// model-space multiscale step: the coarse spline mc [nzc][nxc] evaluated at the fine nodes, mf [nzf][nxf]
cudaError_t launch_spline_refine(const float *zc, int nzc, const float *xc, int nxc, const float *mc, const float *zf,
                                 int nzf, const float *xf, int nxf, float *mf, cudaStream_t st);
// VP conjugate gradients (device scalars)
cudaError_t launch_dot(const float *x, const float *y, long long n, double *partials, int nblocks, double *out,
                       int accumulate, double scale, cudaStream_t st);
cudaError_t launch_dso_add(const float *p, float *hp, int nh, long long PP, float eps2, cudaStream_t st);
cudaError_t launch_axpby_dev(float *y, const float *x, long long n, const double *sc, int ia, float sa, int ib,
                             cudaStream_t st);
cudaError_t launch_cg_scalars(double *sc, int mode, double *history, int k, cudaStream_t st);

// ---- packed two-lane FP32 arithmetic (add/sub/mul/fma.rn.f32x2, sm_100 and later): one instruction
// performs the operation on two independent FP32 values held in a 64-bit register pair, each with
// the rounding of the scalar instruction, so it halves the floating-point issue slots.
typedef unsigned long long f32x2;
__device__ __forceinline__ f32x2 pk(float lo, float hi)
{
    f32x2 r;
    asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(lo), "f"(hi));
    return r;
}
__device__ __forceinline__ void upk(f32x2 v, float &lo, float &hi)
{
    asm("mov.b64 {%0, %1}, %2;" : "=f"(lo), "=f"(hi) : "l"(v));
}
__device__ __forceinline__ f32x2 add2(f32x2 a, f32x2 b)
{
    f32x2 d;
    asm("add.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}
__device__ __forceinline__ f32x2 sub2(f32x2 a, f32x2 b)
{
    f32x2 d;
    asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}
__device__ __forceinline__ f32x2 mul2(f32x2 a, f32x2 b)
{
    f32x2 d;
    asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}
__device__ __forceinline__ f32x2 fma2(f32x2 a, f32x2 b, f32x2 c)
{
    f32x2 d;
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(a), "l"(b), "l"(c));
    return d;
}
__device__ __forceinline__ f32x2 bits(const float2 &v) { return *reinterpret_cast<const f32x2 *>(&v); }

}  // namespace fwk
