// Subsurface-offset extension kernels (Barnier et al., Theory section: Born
// modelling extended with horizontal subsurface offsets, Eq. 1, and its
// adjoint, the extended imaging condition, Eqs. 2-5; tomographic operator,
// Eq. 9).
//
//   scatter    e(y)   = sum_h W(y-h, h) D(y-2h)          (sigma = +1)
//   transpose  z(u)   = sum_h W(u+h, h) L(u+2h)          (sigma = -1)
//   image      I(x,h) += sum_{shots,steps} D(x-h) L(x+h)
//   contract   G(x)   += sum_h p~(x,h) sum D(x-h) L(x+h)
//   local      G(x)   += sum D (alpha L + M2) + Ds L
//
// The weights W = b p~ (nh values per point) are shared by every shot and
// every time step, so these kernels run once per segment of K time steps over
// all K x S (step, shot) pairs of a batch: a CTA owns one row and 128 columns,
// keeps its nh weights (or nh image accumulators) in registers for the whole
// segment, and streams the pairs' D/L rows through a double-buffered
// shared-memory window (global loads of pair p+1 are issued before the
// arithmetic of pair p).  Weight and image traffic is then 1/(K S) of a
// per-step formulation.
#include "fwime_kernels.cuh"

namespace fwk {

__device__ __forceinline__ long long ring_off(const RingRef &r, int n, int j)
{
    const int slot = r.mod > 0 ? (n + r.shift) % r.mod : j + r.shift;
    return (long long)slot * r.slot_stride;
}

// ------------------------------------------------------------------ scatter

template <int NH>
__global__ void __launch_bounds__(EXT_TX) k_scatter(const ExtArgs a)
{
    extern __shared__ float sm[];
    const int nh = NH > 0 ? NH : a.nh;
    const int hm = (nh - 1) / 2;
    const int Z = a.z_lo + blockIdx.y;
    const int y0 = a.x_lo + blockIdx.x * EXT_TX;
    const int y = y0 + threadIdx.x;
    const bool yin = y < a.x_hi;
    const int span = EXT_TX + 4 * hm;
    const int wbase = y0 - 2 * hm;
    const long long rowoff = (long long)Z * a.NXP;
    float *out_base = const_cast<float *>(a.outr.base);

    float Wr[NH > 0 ? NH : 1];
    if (NH > 0) {
#pragma unroll
        for (int ih = 0; ih < (NH > 0 ? NH : 1); ++ih) {
            const int xs = y - a.sigma * (ih - hm);
            Wr[ih] = (yin && xs >= 0 && xs < a.NXP) ? __ldg(a.W + ih * a.P + rowoff + xs) : 0.f;
        }
    }
    constexpr int MAXPF = (EXT_TX + 4 * ((MAX_NH - 1) / 2) + EXT_TX - 1) / EXT_TX;
    const int npf = (span + EXT_TX - 1) / EXT_TX;
    float pre[MAXPF];

    auto load_window = [&](int p) {
        const int j = p / a.S, s = p % a.S, n = a.n0 + j;
        const float *src = a.in.base + ring_off(a.in, n, j) + (long long)s * a.P + rowoff;
#pragma unroll
        for (int k = 0; k < MAXPF; ++k) {
            if (k < npf) {
                const int i = threadIdx.x + k * EXT_TX;
                const int xp = wbase + i;
                pre[k] = (i < span && xp >= 0 && xp < a.NXP) ? __ldg(src + xp) : 0.f;
            }
        }
    };

    if (a.npair > 0) load_window(0);
    for (int p = 0; p < a.npair; ++p) {
        float *buf = sm + (p & 1) * span;
#pragma unroll
        for (int k = 0; k < MAXPF; ++k) {
            const int i = threadIdx.x + k * EXT_TX;
            if (k < npf && i < span) buf[i] = pre[k];
        }
        __syncthreads();
        if (p + 1 < a.npair) load_window(p + 1);
        float acc = 0.f;
        const int c0 = threadIdx.x + 2 * hm;
        if (NH > 0) {
#pragma unroll
            for (int ih = 0; ih < (NH > 0 ? NH : 1); ++ih) acc = fmaf(Wr[ih], buf[c0 - 2 * a.sigma * (ih - hm)], acc);
        } else {
            for (int ih = 0; ih < nh; ++ih) {
                const int xs = y - a.sigma * (ih - hm);
                const float wv = (yin && xs >= 0 && xs < a.NXP) ? __ldg(a.W + ih * a.P + rowoff + xs) : 0.f;
                acc = fmaf(wv, buf[c0 - 2 * a.sigma * (ih - hm)], acc);
            }
        }
        if (yin) {
            const int j = p / a.S, s = p % a.S, n = a.n0 + j;
            float *o = out_base + ring_off(a.outr, n, j) + (long long)s * a.P + rowoff + y;
            *o = a.accumulate ? *o + acc : acc;
        }
    }
}

cudaError_t launch_scatter(const ExtArgs &a, cudaStream_t st)
{
    if (a.npair <= 0 || a.x_hi <= a.x_lo || a.z_hi <= a.z_lo) return cudaSuccess;
    dim3 grid((a.x_hi - a.x_lo + EXT_TX - 1) / EXT_TX, a.z_hi - a.z_lo);
    const int hm = (a.nh - 1) / 2;
    const size_t smem = 2 * (EXT_TX + 4 * hm) * sizeof(float);
    switch (a.nh) {
    case 1: k_scatter<1><<<grid, EXT_TX, smem, st>>>(a); break;
    case 3: k_scatter<3><<<grid, EXT_TX, smem, st>>>(a); break;
    case 5: k_scatter<5><<<grid, EXT_TX, smem, st>>>(a); break;
    case 11: k_scatter<11><<<grid, EXT_TX, smem, st>>>(a); break;
    case 21: k_scatter<21><<<grid, EXT_TX, smem, st>>>(a); break;
    case 31: k_scatter<31><<<grid, EXT_TX, smem, st>>>(a); break;
    case 41: k_scatter<41><<<grid, EXT_TX, smem, st>>>(a); break;
    default: k_scatter<0><<<grid, EXT_TX, smem, st>>>(a); break;
    }
    return cudaGetLastError();
}

// ------------------------------------------------------------------ imaging

template <int NH, int MODE>
__global__ void __launch_bounds__(EXT_TX) k_image(const ImgArgs a)
{
    extern __shared__ float sm[];
    const int nh = NH > 0 ? NH : a.nh;
    const int hm = (nh - 1) / 2;
    const int Z = a.z_lo + blockIdx.y;
    const int x0 = a.x_lo + blockIdx.x * EXT_TX;
    const int X = x0 + threadIdx.x;
    const bool xin = X < a.x_hi;
    const int span = EXT_TX + 2 * hm;
    const int wbase = x0 - hm;
    const long long rowoff = (long long)Z * a.NXP;

    constexpr int NA = (MODE == IMG_EXT && NH > 0) ? NH : 1;
    constexpr int NW = (MODE == IMG_CONTRACT && NH > 0) ? NH : 1;
    float acc[NA];
#pragma unroll
    for (int i = 0; i < NA; ++i) acc[i] = 0.f;
    float ptr[NW];
    if (MODE == IMG_CONTRACT && NH > 0) {
#pragma unroll
        for (int ih = 0; ih < NW; ++ih) ptr[ih] = xin ? __ldg(a.pt + ih * a.P + rowoff + X) : 0.f;
    }
    // generic-nh image accumulators live in shared memory after the windows
    float *gacc = sm + 4 * span;
    if (MODE == IMG_EXT && NH == 0)
        for (int ih = 0; ih < nh; ++ih) gacc[ih * EXT_TX + threadIdx.x] = 0.f;

    constexpr int MAXPF = (EXT_TX + 2 * ((MAX_NH - 1) / 2) + EXT_TX - 1) / EXT_TX;
    const int npf = (span + EXT_TX - 1) / EXT_TX;
    float pd[MAXPF], pl[MAXPF];

    auto load_window = [&](int p) {
        const int j = p / a.S, s = p % a.S, n = a.n0 + j;
        const float *sd = a.D.base + ring_off(a.D, n, j) + (long long)s * a.P + rowoff;
        const float *sl = a.L.base + ring_off(a.L, n, j) + (long long)s * a.P + rowoff;
#pragma unroll
        for (int k = 0; k < MAXPF; ++k) {
            if (k < npf) {
                const int i = threadIdx.x + k * EXT_TX;
                const int xp = wbase + i;
                const bool ok = i < span && xp >= 0 && xp < a.NXP;
                pd[k] = ok ? __ldg(sd + xp) : 0.f;
                pl[k] = ok ? __ldg(sl + xp) : 0.f;
            }
        }
    };

    if (a.npair > 0) load_window(0);
    for (int p = 0; p < a.npair; ++p) {
        float *bd = sm + (p & 1) * 2 * span;
        float *bl = bd + span;
#pragma unroll
        for (int k = 0; k < MAXPF; ++k) {
            const int i = threadIdx.x + k * EXT_TX;
            if (k < npf && i < span) { bd[i] = pd[k]; bl[i] = pl[k]; }
        }
        __syncthreads();
        if (p + 1 < a.npair) load_window(p + 1);
        // D(X - h) at bd[tx + hm - h], L(X + h) at bl[tx + hm + h], h = ih - hm
        const int t = threadIdx.x;
        if (NH > 0) {
            if (MODE == IMG_EXT) {
#pragma unroll
                for (int ih = 0; ih < NA; ++ih) acc[ih] = fmaf(bd[t + 2 * hm - ih], bl[t + ih], acc[ih]);
            } else {
                float s = 0.f;
#pragma unroll
                for (int ih = 0; ih < NW; ++ih) s = fmaf(ptr[ih] * bd[t + 2 * hm - ih], bl[t + ih], s);
                acc[0] += s;
            }
        } else {
            if (MODE == IMG_EXT) {
                for (int ih = 0; ih < nh; ++ih)
                    gacc[ih * EXT_TX + t] = fmaf(bd[t + 2 * hm - ih], bl[t + ih], gacc[ih * EXT_TX + t]);
            } else {
                float s = 0.f;
                for (int ih = 0; ih < nh; ++ih) {
                    const float pv = xin ? __ldg(a.pt + ih * a.P + rowoff + X) : 0.f;
                    s = fmaf(pv * bd[t + 2 * hm - ih], bl[t + ih], s);
                }
                acc[0] += s;
            }
        }
    }
    if (!xin) return;
    if (MODE == IMG_EXT) {
        for (int ih = 0; ih < nh; ++ih) {
            const float v = NH > 0 ? acc[ih < NA ? ih : 0] : gacc[ih * EXT_TX + threadIdx.x];
            a.img[ih * a.P + rowoff + X] += v;
        }
    } else {
        a.img[rowoff + X] += acc[0];
    }
}

// pointwise (h = 0) accumulation: G += sum_pairs D (alpha L + M2) + Ds L
__global__ void __launch_bounds__(EXT_TX) k_image_local(const ImgArgs a)
{
    const int Z = a.z_lo + blockIdx.y;
    const int X = a.x_lo + blockIdx.x * EXT_TX + threadIdx.x;
    if (X >= a.x_hi) return;
    const long long off = (long long)Z * a.NXP + X;
    float acc = 0.f;
    for (int p = 0; p < a.npair; ++p) {
        const int j = p / a.S, s = p % a.S, n = a.n0 + j;
        const long long so = (long long)s * a.P + off;
        const float l = __ldg(a.L.base + ring_off(a.L, n, j) + so);
        float t = a.alpha * l;
        if (a.M2.base) t += __ldg(a.M2.base + ring_off(a.M2, n, j) + so);
        acc = fmaf(__ldg(a.D.base + ring_off(a.D, n, j) + so), t, acc);
        if (a.Ds.base) acc = fmaf(__ldg(a.Ds.base + ring_off(a.Ds, n, j) + so), l, acc);
    }
    a.img[off] += acc;
}

template <int MODE>
static void launch_image_nh(const ImgArgs &a, dim3 grid, size_t smem, cudaStream_t st)
{
    switch (a.nh) {
    case 1: k_image<1, MODE><<<grid, EXT_TX, smem, st>>>(a); break;
    case 3: k_image<3, MODE><<<grid, EXT_TX, smem, st>>>(a); break;
    case 5: k_image<5, MODE><<<grid, EXT_TX, smem, st>>>(a); break;
    case 11: k_image<11, MODE><<<grid, EXT_TX, smem, st>>>(a); break;
    case 21: k_image<21, MODE><<<grid, EXT_TX, smem, st>>>(a); break;
    case 31: k_image<31, MODE><<<grid, EXT_TX, smem, st>>>(a); break;
    case 41: k_image<41, MODE><<<grid, EXT_TX, smem, st>>>(a); break;
    default: k_image<0, MODE><<<grid, EXT_TX, smem, st>>>(a); break;
    }
}

cudaError_t launch_image(const ImgArgs &a, int mode, cudaStream_t st)
{
    if (a.npair <= 0 || a.x_hi <= a.x_lo || a.z_hi <= a.z_lo) return cudaSuccess;
    dim3 grid((a.x_hi - a.x_lo + EXT_TX - 1) / EXT_TX, a.z_hi - a.z_lo);
    if (mode == IMG_LOCAL) {
        k_image_local<<<grid, EXT_TX, 0, st>>>(a);
        return cudaGetLastError();
    }
    const int hm = (a.nh - 1) / 2;
    size_t smem = 4 * (EXT_TX + 2 * hm) * sizeof(float);
    const bool generic = !(a.nh == 1 || a.nh == 3 || a.nh == 5 || a.nh == 11 || a.nh == 21 || a.nh == 31 ||
                           a.nh == 41);
    if (generic && mode == IMG_EXT) {
        smem += (size_t)a.nh * EXT_TX * sizeof(float);
        if (smem > 48 * 1024) {
            cudaError_t e =
                cudaFuncSetAttribute(k_image<0, IMG_EXT>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
            if (e != cudaSuccess) return e;
        }
    }
    if (mode == IMG_EXT) launch_image_nh<IMG_EXT>(a, grid, smem, st);
    else launch_image_nh<IMG_CONTRACT>(a, grid, smem, st);
    return cudaGetLastError();
}

}  // namespace fwk
