// Time-lag extension kernels (Barnier et al., Theory section: Born modelling extended with time lags,
// Eq. 1, and its adjoint, the extended imaging condition, Eqs. 2-5).  Symmetric lags
// tau_i = s_i dt, s_i = (i - hm) L, couple the source side at t - tau with the receiver side at t + tau:
//
//   scatter  e^n(x)    = sum_i W(x, i) D^{n - 2 s_i}(x)           (W = b p~, D^m = 0 outside 0..nt-2)
//   transpose z^m(x)   = sum_i W(x, i) L^{m + 2 s_i}(x)           (sigma = -1: the lag index reversed)
//   image    I(x, i)  += sum_{shots} sum_n D^{n - 2 s_i}(x) L^n(x)
//
// Output step n = base + 2 L j only reads D at steps of the same residue modulo 2L,
// m = base + 2 L (j - i + hm), so a thread that owns one point and JC consecutive outputs of one residue
// class needs the JC + 2 hm samples m_k = base + 2 L (k - hm) of that class: every sample it loads
// serves up to JC (scatter) or nh (image) multiply-adds, with the nh weights or accumulators in
// registers.  Planes of the rings are [S][P]; consecutive threads take consecutive columns of one row
// (coalesced), the time samples of a point are strided by the ring's slot stride.
#include "fwime_kernels.cuh"

namespace fwk {

// packed two-lane FP32 form (f32x2) of the imaging kernel: measured faster (-3.7 % at nh 21); the scatter's
// packed form measured 8.7 % slower (its scalar form keeps JC independent chains per thread) and is not built
#ifndef FWIME_TL_IMG_F32X2
#define FWIME_TL_IMG_F32X2 1
#endif
#ifndef FWIME_TL_IMG_MINB
#define FWIME_TL_IMG_MINB 4   // resident CTAs the imaging kernel is compiled for (up to 21 lags, JC <= 24; spills beyond)
#endif
constexpr int TL_TX = 128;      // threads per CTA (consecutive columns)
#ifndef FWIME_TLI_TX
#define FWIME_TLI_TX 64   // lag imaging: CTAs of one point per thread stream a whole segment, so more and smaller
                          // CTAs fill the last wave better (128 -> 64: 3922 -> 4137 GB/s, 21 lags, 100 shots)
#endif
constexpr int TLI_TX = FWIME_TLI_TX;   // threads per CTA of the lag imaging kernel
// JC, the outputs of one residue class a thread handles (one chunk), is 16, 24 or 32, chosen per
// segment by tlag_jc so that the chunks cover the class's outputs with the fewest wasted window loads

// element offset of time step m in ring r (m >= 0)
__device__ __forceinline__ long long tl_slot(const RingRef &r, int m)
{
    return (long long)((r.mod > 0 ? (m + r.shift) % r.mod : m + r.shift)) * r.slot_stride;
}


// blockIdx.x: column block, blockIdx.y: row, blockIdx.z: shot.  A thread walks the residue classes of its
// point, and the chunks of each class in time order: chunk c's window starts JC samples after chunk
// c - 1's, so the last 2 hm samples of one window are the first of the next and stay in registers.  Every
// sample of a class is loaded once per segment (c + 2 hm loads for c outputs, instead of JC + 2 hm per
// chunk of JC), and the nh weights once per point and shot.
template <int NH, int SIGMA, int JC>
__global__ void __launch_bounds__(TL_TX) k_tlag_scatter(const TlagArgs a)
{
    constexpr int HM = (NH - 1) / 2, NW = JC + 2 * HM;
    // ring offsets of the chunk's window samples and outputs (-1: outside the record / the segment): the
    // same for every thread of the CTA, computed once per chunk into shared memory
    __shared__ long long s_doff[NW], s_eoff[JC];
    const int Z = a.z_lo + blockIdx.y;
    const int step = 2 * a.lag;
    const int s = blockIdx.z;
    const int X = a.x_lo + blockIdx.x * TL_TX + threadIdx.x;
    const bool act = X < a.x_hi;                          // no early exit: the CTA shares barriers
    const long long pp = (long long)Z * a.NXP + (act ? X : a.x_lo), off = (long long)s * a.P + pp;
    float Wr[NH];   // sigma = -1 reads lag i at m + 2 s_i = m - 2 s_(nh-1-i): the weights reversed
#pragma unroll
    for (int i = 0; i < NH; ++i) Wr[i] = __ldg(a.W + (SIGMA > 0 ? i : NH - 1 - i) * a.P + pp);
    const float *db = a.D.base + off;
    float *ob = const_cast<float *>(a.E.base) + off;
    float win[NW];
#pragma unroll 1
    for (int r = 0; r < step; ++r) {
#pragma unroll 1
        for (int base = a.n0 + r, k0 = 0; base < a.n1; base += step * JC, k0 = 2 * HM) {
            const int m0 = base - step * HM;                  // window sample k is step m0 + k (2 L)
            __syncthreads();                                  // every thread is done with the previous tables
            for (int k = threadIdx.x; k < NW + JC; k += TL_TX) {
                if (k < NW) {
                    const int m = m0 + step * k;
                    s_doff[k] = (m >= 0 && m <= a.nt - 2) ? tl_slot(a.D, m) : -1;
                } else {
                    const int n = base + step * (k - NW);
                    s_eoff[k - NW] = n < a.n1 ? tl_slot(a.E, n - a.n0) : -1;
                }
            }
            __syncthreads();
            if (!act) continue;
            if (k0 > 0) {                                     // carried over from the previous chunk
#pragma unroll
                for (int k = 0; k < 2 * HM; ++k) win[k] = win[k + JC];
#pragma unroll
                for (int k = 2 * HM; k < NW; ++k) {
                    const long long o = s_doff[k];
                    win[k] = o >= 0 ? __ldg(db + o) : 0.f;
                }
            } else {
#pragma unroll
                for (int k = 0; k < NW; ++k) {
                    const long long o = s_doff[k];
                    win[k] = o >= 0 ? __ldg(db + o) : 0.f;
                }
            }
            float acc[JC];
#pragma unroll
            for (int j = 0; j < JC; ++j) acc[j] = 0.f;
#pragma unroll
            for (int j = 0; j < JC; ++j)
#pragma unroll
                for (int i = 0; i < NH; ++i) acc[j] = fmaf(Wr[i], win[j - i + 2 * HM], acc[j]);
#pragma unroll
            for (int j = 0; j < JC; ++j) {
                const long long eo = s_eoff[j];
                if (eo >= 0) {
                    float *o = ob + eo;
                    *o = a.accumulate ? *o + acc[j] : acc[j];
                }
            }
        }
    }
}

// generic nh: weights and samples re-read per output (any odd nh)
__global__ void __launch_bounds__(TL_TX) k_tlag_scatter_gen(const TlagArgs a)
{
    const int X = a.x_lo + blockIdx.x * TL_TX + threadIdx.x;
    if (X >= a.x_hi) return;
    const int Z = a.z_lo + blockIdx.y;
    const int r = blockIdx.z % (2 * a.lag), s = blockIdx.z / (2 * a.lag);   // (shot, residue)
    const long long pp = (long long)Z * a.NXP + X, off = (long long)s * a.P + pp;
    const int hm = (a.nh - 1) / 2;
    for (int n = a.n0 + r; n < a.n1; n += 2 * a.lag) {   // the residue class's outputs
        float acc = 0.f;
        for (int i = 0; i < a.nh; ++i) {
            const int m = n - a.sigma * 2 * a.lag * (i - hm);
            if (m >= 0 && m <= a.nt - 2)
                acc = fmaf(__ldg(a.W + i * a.P + pp), __ldg(a.D.base + tl_slot(a.D, m) + off), acc);
        }
        float *o = const_cast<float *>(a.E.base) + tl_slot(a.E, n - a.n0) + off;
        *o = a.accumulate ? *o + acc : acc;
    }
}

// blockIdx.x: column block, blockIdx.y: row; the thread walks shots, residues and chunks.  The ring
// offsets of a (residue, chunk)'s window and receiver-side samples are the same for every thread of the
// CTA: computed once per iteration into shared memory.  Within a residue class the chunks' windows
// overlap by 2 hm samples, carried over in registers (each D sample loaded once per class and segment).
template <int NH, int JC>
__global__ void __launch_bounds__(TLI_TX, (NH <= 21 && JC <= 24) ? FWIME_TL_IMG_MINB * 128 / TLI_TX : 1)
    k_tlag_image(const TlagArgs a)
{
    constexpr int HM = (NH - 1) / 2, NW = JC + 2 * HM;
    __shared__ long long s_doff[NW], s_loff[JC];
    const int X = a.x_lo + blockIdx.x * TLI_TX + threadIdx.x;
    const bool act = X < a.x_hi;                          // no early exit: the CTA shares barriers
    const int Z = a.z_lo + blockIdx.y;
    const long long pp = (long long)Z * a.NXP + (act ? X : a.x_lo);
    const int step = 2 * a.lag;
    float acc[NH];
#pragma unroll
    for (int i = 0; i < NH; ++i) acc[i] = 0.f;
#if FWIME_TL_IMG_F32X2
    // Packed form: sample j contributes win[k] lv[j], k = j - i + 2 HM, to lag i.  For even j the lag
    // pairs (2q + 1, 2q + 2) read the aligned sample pairs (k - 1, k) (k - 1 even) and lag 0 stays
    // scalar; for odd j the lag pairs (2q, 2q + 1) do and lag NH - 1 stays scalar.  A register pair
    // holds (lag i + 1, lag i); the two sets are added at the end.
    f32x2 pe[HM > 0 ? HM : 1], po[HM > 0 ? HM : 1];
    float se = 0.f, so = 0.f;
#pragma unroll
    for (int q = 0; q < HM; ++q) pe[q] = po[q] = pk(0.f, 0.f);
#endif
    float win[NW];                                        // the chunk's window of one residue class
#pragma unroll 1
    for (int s = 0; s < a.S; ++s) {
        const long long off = (long long)s * a.P + pp;
#pragma unroll 1
        for (int r = 0; r < step; ++r) {
#pragma unroll 1
            for (int base = a.n0 + r, k0 = 0; base < a.n1; base += step * JC, k0 = 2 * HM) {
                const int m0 = base - step * HM;
                __syncthreads();                          // every thread is done with the previous tables
                for (int k = threadIdx.x; k < NW + JC; k += TLI_TX) {
                    if (k < NW) {
                        const int m = m0 + step * k;
                        s_doff[k] = (m >= 0 && m <= a.nt - 2) ? tl_slot(a.D, m) : -1;
                    } else {
                        const int n = base + step * (k - NW);
                        s_loff[k - NW] = n < a.n1 ? tl_slot(a.L, n) : -1;
                    }
                }
                __syncthreads();
                if (!act) continue;
                float lv[JC];
                const float *db = a.D.base + off, *lb0 = a.L.base + off;
                if (k0 > 0) {                             // carried over from the previous chunk
#pragma unroll
                    for (int k = 0; k < 2 * HM; ++k) win[k] = win[k + JC];
#pragma unroll
                    for (int k = 2 * HM; k < NW; ++k) {
                        const long long o = s_doff[k];
                        win[k] = o >= 0 ? __ldg(db + o) : 0.f;
                    }
                } else {
#pragma unroll
                    for (int k = 0; k < NW; ++k) {
                        const long long o = s_doff[k];
                        win[k] = o >= 0 ? __ldg(db + o) : 0.f;
                    }
                }
#pragma unroll
                for (int j = 0; j < JC; ++j) {
                    const long long o = s_loff[j];
                    lv[j] = o >= 0 ? __ldg(lb0 + o) : 0.f;
                }
#if FWIME_TL_IMG_F32X2
#pragma unroll
                for (int j = 0; j < JC; ++j) {
                    const f32x2 lb = pk(lv[j], lv[j]);
                    if (j % 2 == 0) {
#pragma unroll
                        for (int q = 0; q < HM; ++q) {
                            const int k = j - (2 * q + 1) + 2 * HM;
                            pe[q] = fma2(pk(win[k - 1], win[k]), lb, pe[q]);
                        }
                        se = fmaf(win[j + 2 * HM], lv[j], se);
                    } else {
#pragma unroll
                        for (int q = 0; q < HM; ++q) {
                            const int k = j - 2 * q + 2 * HM;
                            po[q] = fma2(pk(win[k - 1], win[k]), lb, po[q]);
                        }
                        so = fmaf(win[j], lv[j], so);
                    }
                }
#else
#pragma unroll
                for (int i = 0; i < NH; ++i)
#pragma unroll
                    for (int j = 0; j < JC; ++j) acc[i] = fmaf(win[j - i + 2 * HM], lv[j], acc[i]);
#endif
            }
        }
    }
#if FWIME_TL_IMG_F32X2
    {
        float ve[NH], vo[NH];
        ve[0] = se;
        vo[NH - 1] = so;
#pragma unroll
        for (int q = 0; q < HM; ++q) {
            upk(pe[q], ve[2 * q + 2], ve[2 * q + 1]);
            upk(po[q], vo[2 * q + 1], vo[2 * q]);
        }
#pragma unroll
        for (int i = 0; i < NH; ++i) acc[i] = ve[i] + vo[i];
    }
#endif
    if (!act) return;
#pragma unroll
    for (int i = 0; i < NH; ++i) a.img[i * a.P + pp] += acc[i];
}

__global__ void __launch_bounds__(TL_TX) k_tlag_image_gen(const TlagArgs a)
{
    const int X = a.x_lo + blockIdx.x * TL_TX + threadIdx.x;
    if (X >= a.x_hi) return;
    const int Z = a.z_lo + blockIdx.y;
    const long long pp = (long long)Z * a.NXP + X;
    const int hm = (a.nh - 1) / 2;
    for (int i = 0; i < a.nh; ++i) {
        float acc = 0.f;
        for (int s = 0; s < a.S; ++s) {
            const long long off = (long long)s * a.P + pp;
            for (int n = a.n0; n < a.n1; ++n) {
                const int m = n - 2 * a.lag * (i - hm);
                if (m >= 0 && m <= a.nt - 2)
                    acc = fmaf(__ldg(a.D.base + tl_slot(a.D, m) + off), __ldg(a.L.base + tl_slot(a.L, n) + off), acc);
            }
        }
        a.img[i * a.P + pp] += acc;
    }
}

template <int NH, int JC>
static void launch_tlag_scatter_jc(const TlagArgs &a, dim3 grid, cudaStream_t st)
{
    if (a.sigma > 0) k_tlag_scatter<NH, 1, JC><<<grid, TL_TX, 0, st>>>(a);
    else k_tlag_scatter<NH, -1, JC><<<grid, TL_TX, 0, st>>>(a);
}
template <int NH>
static void launch_tlag_scatter_nh(const TlagArgs &a, dim3 grid, cudaStream_t st)
{
    if (a.jc == 20) launch_tlag_scatter_jc<NH, 20>(a, grid, st);
    else if (a.jc == 24) launch_tlag_scatter_jc<NH, 24>(a, grid, st);
    else if (a.jc == 32) launch_tlag_scatter_jc<NH, 32>(a, grid, st);
    else launch_tlag_scatter_jc<NH, 16>(a, grid, st);
}

cudaError_t launch_tlag_scatter(const TlagArgs &a, cudaStream_t st)
{
    if (a.n1 <= a.n0 || a.x_hi <= a.x_lo || a.z_hi <= a.z_lo) return cudaSuccess;
    if (a.jc != 16 && a.jc != 20 && a.jc != 24 && a.jc != 32) return cudaErrorInvalidValue;
    // generic nh: one thread per (point, shot, residue); templated: per (point, shot)
    const bool gen = a.nh != 1 && a.nh != 3 && a.nh != 5 && a.nh != 11 && a.nh != 21 && a.nh != 31 && a.nh != 41;
    dim3 grid((a.x_hi - a.x_lo + TL_TX - 1) / TL_TX, a.z_hi - a.z_lo, a.S * (gen ? 2 * a.lag : 1));
    switch (a.nh) {
    case 1: launch_tlag_scatter_nh<1>(a, grid, st); break;
    case 3: launch_tlag_scatter_nh<3>(a, grid, st); break;
    case 5: launch_tlag_scatter_nh<5>(a, grid, st); break;
    case 11: launch_tlag_scatter_nh<11>(a, grid, st); break;
    case 21: launch_tlag_scatter_nh<21>(a, grid, st); break;
    case 31: launch_tlag_scatter_nh<31>(a, grid, st); break;
    case 41: launch_tlag_scatter_nh<41>(a, grid, st); break;
    default: k_tlag_scatter_gen<<<grid, TL_TX, 0, st>>>(a);
    }
    return cudaGetLastError();
}

template <int NH>
static void launch_tlag_image_nh(const TlagArgs &a, dim3 grid, cudaStream_t st)
{
    if (a.jc == 20) k_tlag_image<NH, 20><<<grid, TLI_TX, 0, st>>>(a);
    else if (a.jc == 24) k_tlag_image<NH, 24><<<grid, TLI_TX, 0, st>>>(a);
    else if (a.jc == 32) k_tlag_image<NH, 32><<<grid, TLI_TX, 0, st>>>(a);
    else k_tlag_image<NH, 16><<<grid, TLI_TX, 0, st>>>(a);
}

cudaError_t launch_tlag_image(const TlagArgs &a, cudaStream_t st)
{
    if (a.n1 <= a.n0 || a.x_hi <= a.x_lo || a.z_hi <= a.z_lo) return cudaSuccess;
    if (a.jc != 16 && a.jc != 20 && a.jc != 24 && a.jc != 32) return cudaErrorInvalidValue;
    dim3 grid((a.x_hi - a.x_lo + TLI_TX - 1) / TLI_TX, a.z_hi - a.z_lo);
    dim3 grid_gen((a.x_hi - a.x_lo + TL_TX - 1) / TL_TX, a.z_hi - a.z_lo);
    switch (a.nh) {
    case 1: launch_tlag_image_nh<1>(a, grid, st); break;
    case 3: launch_tlag_image_nh<3>(a, grid, st); break;
    case 5: launch_tlag_image_nh<5>(a, grid, st); break;
    case 11: launch_tlag_image_nh<11>(a, grid, st); break;
    case 21: launch_tlag_image_nh<21>(a, grid, st); break;
    case 31: launch_tlag_image_nh<31>(a, grid, st); break;
    case 41: launch_tlag_image_nh<41>(a, grid, st); break;
    default: k_tlag_image_gen<<<grid_gen, TL_TX, 0, st>>>(a);
    }
    return cudaGetLastError();
}

// A segment of K steps holds at most c = ceil(K / 2L) outputs of one residue class.  The kernels load
// each window sample of a class once (c + 2 hm loads, whatever JC), so JC only sets the outputs computed
// past c in the last chunk: the JC with the fewest, ties to the shorter chunk (fewer registers: the
// imaging kernel at nh 21 spills with JC = 24 under its 128-register bound).
int tlag_jc(int K, int lag, int nh)
{
    (void)nh;
    const int c = (K + 2 * lag - 1) / (2 * lag);
    int best = 16;
    long long bc = -1;
    for (const int jc : {16, 20, 24, 32}) {
        const long long padded = (long long)((c + jc - 1) / jc) * jc;
        if (bc < 0 || padded < bc) { bc = padded; best = jc; }
    }
    return best;
}

}  // namespace fwk
