// Model preparation and small elementwise / reduction kernels of libfwime.
#include "fwime_kernels.cuh"

namespace fwk {

// Cerjan-type taper of the Marmousi2 section's absorbing boundary:
// g1(k) = exp(-(0.3 k / W)^2), k = points outside the physical region.
__device__ __forceinline__ float taper1(int k, int W)
{
    if (k == 0 || W == 0) return 1.f;
    const float a = 0.3f * (float)k / (float)W;
    return expf(-a * a);
}

__device__ __forceinline__ int outside(int I, int o, int n)
{
    return I < o ? o - I : (I > o + n - 1 ? I - (o + n - 1) : 0);
}

// c = v^2 dt^2 on the padded grid (v edge-replicated), b = 2/v^3 on the physical
// grid (zero-embedded), 1-D sponge factors (zero on the 4-point halo and on the
// pitch columns), and a CFL / positivity check latched in the status word.
__global__ void k_prep(const PrepArgs a)
{
    const int IX = blockIdx.x * blockDim.x + threadIdx.x;
    const int IZ = blockIdx.y;
    if (IX >= a.NXP) return;
    const bool act = IZ >= 4 && IZ < a.NZ - 4 && IX >= 4 && IX < a.NX - 4;
    const int iz = min(max(IZ - a.o, 0), a.nz - 1), ix = min(max(IX - a.o, 0), a.nx - 1);
    const float vv = a.v[(long long)iz * a.nx + ix];
    const long long p = (long long)IZ * a.NXP + IX;
    // free surface: no sponge on top, the 4 mirror rows above the surface row are rewritten after every
    // step, rows further up are inactive; c = 0 on the surface row (nothing is injected there)
    const bool dead = a.fs && (IZ < a.o - 4 || IZ == a.o);
    a.c[p] = act && !dead ? vv * vv * a.dt * a.dt : 0.f;
    const bool phys = IZ >= a.o && IZ < a.o + a.nz && IX >= a.o && IX < a.o + a.nx;
    a.bpad[p] = phys ? 2.f / (vv * vv * vv) : 0.f;
    if (phys && !(vv > 0.f && vv * vv < a.cfl_limit2)) atomicOr(a.status, ST_CFL);
    if (IZ == 0) a.gx[IX] = (IX >= 4 && IX < a.NX - 4) ? taper1(outside(IX, a.o, a.nx), a.W) : 0.f;
    if (IX == 0)
        a.gz[IZ] = (IZ >= 4 && IZ < a.NZ - 4 && !(a.fs && IZ < a.o - 4))
                       ? ((a.fs && IZ < a.o) ? 1.f : taper1(outside(IZ, a.o, a.nz), a.W))
                       : 0.f;
}

// free surface (pressure release at the top physical row IZ = o): after a step, q = 0 on the surface row
// and the 4 rows above hold the odd mirror -q of the 4 rows below; D2t is 0 on the surface row
__global__ void k_free_surface(float *q, float *d2, long long P, int NXP, int o)
{
    const int IX = blockIdx.x * blockDim.x + threadIdx.x;
    if (IX >= NXP) return;
    const long long f = (long long)blockIdx.y * P + IX;
    q[f + (long long)o * NXP] = 0.f;
#pragma unroll
    for (int k = 1; k <= 4; ++k) q[f + (long long)(o - k) * NXP] = -q[f + (long long)(o + k) * NXP];
    if (d2) d2[f + (long long)o * NXP] = 0.f;
}

cudaError_t launch_free_surface(float *q, float *d2, int nshot, long long P, int NXP, int o, cudaStream_t st)
{
    k_free_surface<<<dim3((NXP + 127) / 128, nshot), 128, 0, st>>>(q, d2, P, NXP, o);
    return cudaGetLastError();
}

cudaError_t launch_prep(const PrepArgs &a, cudaStream_t st)
{
    dim3 grid((a.NXP + 127) / 128, a.NZ);
    k_prep<<<grid, 128, 0, st>>>(a);
    return cudaGetLastError();
}

// out_pad = alpha * scale_pad * embed(phys)  (scale_pad may be null = 1)
__global__ void k_embed_scale(const float *phys, const float *scale_pad, float *out_pad, int nz, int nx, int o,
                              int NXP, float alpha)
{
    const int ix = blockIdx.x * blockDim.x + threadIdx.x, iz = blockIdx.y;
    if (ix >= nx) return;
    const long long p = (long long)(iz + o) * NXP + ix + o;
    const float s = scale_pad ? scale_pad[p] : 1.f;
    out_pad[p] = alpha * s * phys[(long long)iz * nx + ix];
}

cudaError_t launch_embed_scale(const float *phys, const float *scale_pad, float *out_pad, int nz, int nx, int o,
                               int NXP, float alpha, cudaStream_t st)
{
    dim3 grid((nx + 127) / 128, nz);
    k_embed_scale<<<grid, 128, 0, st>>>(phys, scale_pad, out_pad, nz, nx, o, NXP, alpha);
    return cudaGetLastError();
}

// Extended weights on the padded grid, one plane per offset:
//   mode 0: W  = b p~               (scattering weights of B~)
//   mode 1: W' = (-3 dv / v) b p~   (db/dv term of T)
//   mode 2: p~ embedded             (contraction of the tomographic adjoint)
__global__ void k_ext_weights(const float *pt, const float *bpad, const float *dv, const float *v, float *Wout, int nz,
                              int nx, int o, int NXP, long long P, int mode)
{
    const int ix = blockIdx.x * blockDim.x + threadIdx.x, iz = blockIdx.y, ih = blockIdx.z;
    if (ix >= nx) return;
    const long long pp = (long long)iz * nx + ix;
    const long long p = (long long)(iz + o) * NXP + ix + o;
    const float pv = pt[(long long)ih * nz * nx + pp];
    float wv;
    if (mode == 0) wv = bpad[p] * pv;
    else if (mode == 1) wv = (-3.f * dv[pp] / v[pp]) * (bpad[p] * pv);
    else wv = pv;
    Wout[(long long)ih * P + p] = wv;
}

cudaError_t launch_ext_weights(const float *pt, const float *bpad, const float *dv, const float *v, float *Wout, int nh,
                               int nz, int nx, int o, int NXP, long long P, int mode, cudaStream_t st)
{
    dim3 grid((nx + 127) / 128, nz, nh);
    k_ext_weights<<<grid, 128, 0, st>>>(pt, bpad, dv, v, Wout, nz, nx, o, NXP, P, mode);
    return cudaGetLastError();
}

// Model-space outputs on the physical grid:
//   mode 0: out[k] (=,+=) b * acc1[k]                                  (B*, B~*: image planes k)
//   mode 1: out    (=,+=) b * acc1 - 3 b / v * sum_h p~[h] acc2[h]        (T*, gradient; acc2 holds the
//                                                                         extended image planes)
__global__ void k_finalize(const float *acc1, const float *acc2, const float *bpad, const float *v, float *out, int nz,
                           int nx, int o, int NXP, long long P, int mode, int accumulate, const float *pt, int nh)
{
    const int ix = blockIdx.x * blockDim.x + threadIdx.x, iz = blockIdx.y, k = blockIdx.z;
    if (ix >= nx) return;
    const long long pp = (long long)iz * nx + ix;
    const long long p = (long long)(iz + o) * NXP + ix + o;
    const float b = bpad[p];
    float val = b * acc1[(long long)k * P + p];
    if (mode == 1) {
        float c = 0.f;
        for (int ih = 0; ih < nh; ++ih) c = fmaf(pt[(long long)ih * nz * nx + pp], acc2[(long long)ih * P + p], c);
        val -= 3.f * b / v[pp] * c;
    }
    float *dst = out + (long long)k * nz * nx + pp;
    *dst = accumulate ? *dst + val : val;
}

cudaError_t launch_finalize(const float *acc1, const float *acc2, const float *bpad, const float *v, float *out,
                            int nplanes, int nz, int nx, int o, int NXP, long long P, int mode, int accumulate,
                            cudaStream_t st, const float *pt, int nh)
{
    dim3 grid((nx + 127) / 128, nz, nplanes);
    k_finalize<<<grid, 128, 0, st>>>(acc1, acc2, bpad, v, out, nz, nx, o, NXP, P, mode, accumulate, pt, nh);
    return cudaGetLastError();
}

// r = pred - dobs and per-block partial sums of r^2 / 2 (FP64, fixed order)
__global__ void k_residual(const float *pred, const float *dobs, float *r, long long n, double *partials)
{
    __shared__ double red[256];
    double acc = 0.0;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const float d = pred[i] - dobs[i];
        r[i] = d;
        acc += 0.5 * (double)d * (double)d;
    }
    red[threadIdx.x] = acc;
    __syncthreads();
    for (int s = blockDim.x / 2; s > 0; s >>= 1) {
        if (threadIdx.x < s) red[threadIdx.x] += red[threadIdx.x + s];
        __syncthreads();
    }
    if (threadIdx.x == 0) partials[blockIdx.x] = red[0];
}

cudaError_t launch_residual(const float *pred, const float *dobs, float *r, long long n, double *partials, int nblocks,
                            cudaStream_t st)
{
    k_residual<<<nblocks, 256, 0, st>>>(pred, dobs, r, n, partials);
    return cudaGetLastError();
}

// sum of the weighted squares sum_h ((|ih - hm| + 1) p~)^2 (the DSO reading), partials per block
__global__ void k_dso(const float *pt, int nh, long long PP, double *partials)
{
    __shared__ double red[256];
    const int hm = (nh - 1) / 2;
    double acc = 0.0;
    const long long n = (long long)nh * PP;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const int ih = (int)(i / PP);
        const double w = (double)abs(ih - hm) + 1.0;
        const double t = w * (double)pt[i];
        acc += t * t;
    }
    red[threadIdx.x] = acc;
    __syncthreads();
    for (int s = blockDim.x / 2; s > 0; s >>= 1) {
        if (threadIdx.x < s) red[threadIdx.x] += red[threadIdx.x + s];
        __syncthreads();
    }
    if (threadIdx.x == 0) partials[blockIdx.x] = red[0];
}

cudaError_t launch_dso(const float *pt, int nh, long long PP, double *partials, int nblocks, cudaStream_t st)
{
    k_dso<<<nblocks, 256, 0, st>>>(pt, nh, PP, partials);
    return cudaGetLastError();
}

// *out (=,+=) sum of partials, in index order (single thread: deterministic)
__global__ void k_sum_partials(const double *partials, int n, double *out, int accumulate, double scale)
{
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    double s = 0.0;
    for (int i = 0; i < n; ++i) s += partials[i];
    *out = accumulate ? *out + scale * s : scale * s;
}

cudaError_t launch_sum_partials(const double *partials, int n, double *out, int accumulate, double scale,
                                cudaStream_t st)
{
    k_sum_partials<<<1, 32, 0, st>>>(partials, n, out, accumulate, scale);
    return cudaGetLastError();
}

__global__ void k_copy(float4 *dst, const float4 *src, long long n4)
{
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n4; i += (long long)gridDim.x * blockDim.x)
        dst[i] = src[i];
}

// device-to-device copy of whole fields (n a multiple of 4 floats, 16-byte aligned)
cudaError_t launch_copy_fields(float *dst, const float *src, long long n, cudaStream_t st)
{
    const long long n4 = n / 4;
    int nb = (int)((n4 + 255) / 256);
    if (nb > 152 * 16) nb = 152 * 16;
    if (nb < 1) nb = 1;
    k_copy<<<nb, 256, 0, st>>>(reinterpret_cast<float4 *>(dst), reinterpret_cast<const float4 *>(src), n4);
    return cudaGetLastError();
}

}  // namespace fwk

// ------------------------------------------------------------ VP conjugate gradients
// Vector kernels of the linear conjugate-gradient solve of the variable projection step
// (Theory section, Eqs. 2-5).  Scalars live in device memory (sc[]) so an iteration never
// waits on the host.  Layout of sc: 0 rr, 1 pHp, 2 alpha, 3 beta, 4 rr_new, 5 phi.

namespace {
__device__ __forceinline__ double block_sum(double v)
{
    __shared__ double red[256];
    red[threadIdx.x] = v;
    __syncthreads();
    for (int s = blockDim.x / 2; s > 0; s >>= 1) {
        if (threadIdx.x < s) red[threadIdx.x] += red[threadIdx.x + s];
        __syncthreads();
    }
    return red[0];
}
}  // namespace

// partials[b] = sum over this block's share of x . y (FP64, fixed order)
__global__ void k_dot(const float *x, const float *y, long long n, double *partials)
{
    double acc = 0.0;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        acc += (double)x[i] * (double)y[i];
    const double s = block_sum(acc);
    if (threadIdx.x == 0) partials[blockIdx.x] = s;
}

// Hp += eps^2 D^2 p with D = diag(|ih - hm| + 1), planes of PP points
__global__ void k_dso_add(const float *p, float *hp, int nh, long long PP, float eps2)
{
    const long long n = (long long)nh * PP;
    const int hm = (nh - 1) / 2;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const float wd = (float)(abs((int)(i / PP) - hm) + 1);
        hp[i] = fmaf(eps2 * wd * wd, p[i], hp[i]);
    }
}

// y = a x + b y with a, b read from device scalars (sign applied): ya = +/- sc[ia], yb = sc[ib] or 1
__global__ void k_axpby_dev(float *y, const float *x, long long n, const double *sc, int ia, float sa, int ib)
{
    const float a = sa * (float)sc[ia];
    const float b = ib >= 0 ? (float)sc[ib] : 1.f;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        y[i] = fmaf(a, x[i], b * y[i]);
}

// scalar updates: mode 0 (after pHp): alpha = rr / pHp, phi -= alpha rr / 2, store the history entry;
// mode 1 (after rr_new): beta = rr_new / rr, rr = rr_new
__global__ void k_cg_scalars(double *sc, int mode, double *history, int k)
{
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    if (mode == 0) {
        sc[2] = sc[1] > 0.0 ? sc[0] / sc[1] : 0.0;
        sc[5] -= 0.5 * sc[2] * sc[0];
        if (history) history[k] = sc[5];
    } else {
        sc[3] = sc[0] > 0.0 ? sc[4] / sc[0] : 0.0;
        sc[0] = sc[4];
    }
}

namespace fwk {
cudaError_t launch_dot(const float *x, const float *y, long long n, double *partials, int nblocks, double *out,
                       int accumulate, double scale, cudaStream_t st)
{
    k_dot<<<nblocks, 256, 0, st>>>(x, y, n, partials);
    return launch_sum_partials(partials, nblocks, out, accumulate, scale, st);
}
cudaError_t launch_dso_add(const float *p, float *hp, int nh, long long PP, float eps2, cudaStream_t st)
{
    k_dso_add<<<1216, 256, 0, st>>>(p, hp, nh, PP, eps2);
    return cudaGetLastError();
}
cudaError_t launch_axpby_dev(float *y, const float *x, long long n, const double *sc, int ia, float sa, int ib,
                             cudaStream_t st)
{
    k_axpby_dev<<<1216, 256, 0, st>>>(y, x, n, sc, ia, sa, ib);
    return cudaGetLastError();
}
cudaError_t launch_cg_scalars(double *sc, int mode, double *history, int k, cudaStream_t st)
{
    k_cg_scalars<<<1, 32, 0, st>>>(sc, mode, history, k);
    return cudaGetLastError();
}
}  // namespace fwk
