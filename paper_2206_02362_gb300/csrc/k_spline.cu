// Linear spline re-parametrisation of the model (Barnier et al., Theory section, Eq. 1: the model m
// lives on a coarse spline grid and the wave equation sees v = S m on the finite-difference grid; the
// gradient of Eqs. 7-9 is mapped back with S*).  Nodes zs[nzs] x xs[nxs] (metres, strictly increasing);
// the physical grid point (iz, ix) sits at (iz dz, ix dx).  Between nodes k and k+1 a point takes the
// weights 1 - a and a, a = (c - node_k) / (node_k+1 - node_k); beyond the end nodes it takes the end
// node's value.  S is a gather per grid point; S* is two gathers (along x, then along z) over the
// support of each node, so every output has one writer and a fixed summation order.
#include "fwime_kernels.cuh"

namespace fwk {

// interval k of coordinate c (nodes[k] <= c < nodes[k+1]) and its weight a; before the first node
// k = 0, a = 0; at or after the last k = n - 2, a = 1; a single node: k = 0, a = 0
__device__ __forceinline__ void spline_locate(const float *nodes, int n, float c, int &k, float &a)
{
    if (n == 1 || c <= nodes[0]) {
        k = 0;
        a = 0.f;
        return;
    }
    if (c >= nodes[n - 1]) {
        k = n - 2;
        a = 1.f;
        return;
    }
    int lo = 0, hi = n - 1;   // nodes[lo] <= c < nodes[hi]
    while (hi - lo > 1) {
        const int mid = (lo + hi) >> 1;
        if (nodes[mid] <= c) lo = mid;
        else hi = mid;
    }
    k = lo;
    a = (c - nodes[lo]) / (nodes[lo + 1] - nodes[lo]);
}

// weight of node l at coordinate c
__device__ __forceinline__ float spline_weight(const float *nodes, int n, float c, int l)
{
    int k;
    float a;
    spline_locate(nodes, n, c, k, a);
    if (n == 1) return l == 0 ? 1.f : 0.f;
    return (k == l ? 1.f - a : 0.f) + (k + 1 == l ? a : 0.f);
}

// grid points whose weight for node l may be non-zero: [lo, hi]
__device__ __forceinline__ void spline_support(const float *nodes, int n, float h, int npts, int l, int &lo, int &hi)
{
    lo = l == 0 ? 0 : (int)floorf(nodes[l - 1] / h);
    hi = l == n - 1 ? npts - 1 : (int)ceilf(nodes[l + 1] / h);
    lo = lo < 0 ? 0 : lo;
    hi = hi > npts - 1 ? npts - 1 : hi;
}

__global__ void k_spline_fwd(const float *zs, int nzs, const float *xs, int nxs, int nz, int nx, float dz, float dx,
                             const float *m, float *v, int accumulate)
{
    const int ix = blockIdx.x * blockDim.x + threadIdx.x, iz = blockIdx.y;
    if (ix >= nx) return;
    int kz, kx;
    float az, ax;
    spline_locate(zs, nzs, (float)iz * dz, kz, az);
    spline_locate(xs, nxs, (float)ix * dx, kx, ax);
    const int kz1 = kz + 1 < nzs ? kz + 1 : kz, kx1 = kx + 1 < nxs ? kx + 1 : kx;
    const float top = (1.f - ax) * m[(long long)kz * nxs + kx] + ax * m[(long long)kz * nxs + kx1];
    const float bot = (1.f - ax) * m[(long long)kz1 * nxs + kx] + ax * m[(long long)kz1 * nxs + kx1];
    const float r = (1.f - az) * top + az * bot;
    float *o = v + (long long)iz * nx + ix;
    *o = accumulate ? *o + r : r;
}

// S* along x: t[iz][l] = sum_ix w_l(x_ix) g[iz][ix]
__global__ void k_spline_adj_x(const float *xs, int nxs, int nz, int nx, float dx, const float *g, float *t)
{
    const int l = blockIdx.x * blockDim.x + threadIdx.x, iz = blockIdx.y;
    if (l >= nxs) return;
    int lo, hi;
    spline_support(xs, nxs, dx, nx, l, lo, hi);
    float s = 0.f;
    for (int ix = lo; ix <= hi; ++ix) s = fmaf(spline_weight(xs, nxs, (float)ix * dx, l), g[(long long)iz * nx + ix], s);
    t[(long long)iz * nxs + l] = s;
}

// S* along z: m[k][l] (=, or +=) sum_iz w_k(z_iz) t[iz][l]
__global__ void k_spline_adj_z(const float *zs, int nzs, int nxs, int nz, float dz, const float *t, float *m,
                               int accumulate)
{
    const int l = blockIdx.x * blockDim.x + threadIdx.x, k = blockIdx.y;
    if (l >= nxs) return;
    int lo, hi;
    spline_support(zs, nzs, dz, nz, k, lo, hi);
    float s = 0.f;
    for (int iz = lo; iz <= hi; ++iz) s = fmaf(spline_weight(zs, nzs, (float)iz * dz, k), t[(long long)iz * nxs + l], s);
    float *o = m + (long long)k * nxs + l;
    *o = accumulate ? *o + s : s;
}

// model-space multiscale step: mf[i][j] = the coarse linear spline of mc at the fine node (zf[i], xf[j])
__global__ void k_spline_refine(const float *zc, int nzc, const float *xc, int nxc, const float *mc, const float *zf,
                                int nzf, const float *xf, int nxf, float *mf)
{
    const int j = blockIdx.x * blockDim.x + threadIdx.x, i = blockIdx.y;
    if (j >= nxf) return;
    int kz, kx;
    float az, ax;
    spline_locate(zc, nzc, zf[i], kz, az);
    spline_locate(xc, nxc, xf[j], kx, ax);
    const int kz1 = kz + 1 < nzc ? kz + 1 : kz, kx1 = kx + 1 < nxc ? kx + 1 : kx;
    const float top = (1.f - ax) * mc[(long long)kz * nxc + kx] + ax * mc[(long long)kz * nxc + kx1];
    const float bot = (1.f - ax) * mc[(long long)kz1 * nxc + kx] + ax * mc[(long long)kz1 * nxc + kx1];
    mf[(long long)i * nxf + j] = (1.f - az) * top + az * bot;
}

cudaError_t launch_spline_refine(const float *zc, int nzc, const float *xc, int nxc, const float *mc, const float *zf,
                                 int nzf, const float *xf, int nxf, float *mf, cudaStream_t st)
{
    k_spline_refine<<<dim3((nxf + 127) / 128, nzf), 128, 0, st>>>(zc, nzc, xc, nxc, mc, zf, nzf, xf, nxf, mf);
    return cudaGetLastError();
}

cudaError_t launch_spline(const float *zs, int nzs, const float *xs, int nxs, int nz, int nx, float dz, float dx,
                          const float *in, float *out, float *tmp, int adjoint, int accumulate, cudaStream_t st)
{
    if (!adjoint) {
        k_spline_fwd<<<dim3((nx + 127) / 128, nz), 128, 0, st>>>(zs, nzs, xs, nxs, nz, nx, dz, dx, in, out, accumulate);
        return cudaGetLastError();
    }
    k_spline_adj_x<<<dim3((nxs + 63) / 64, nz), 64, 0, st>>>(xs, nxs, nz, nx, dx, in, tmp);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    k_spline_adj_z<<<dim3((nxs + 63) / 64, nzs), 64, 0, st>>>(zs, nzs, nxs, nz, dz, tmp, out, accumulate);
    return cudaGetLastError();
}

}  // namespace fwk
