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

// Walks the (step, shot) pairs of a segment in order p = 0, 1, ... (shot fastest) without
// integer division: pointer to the pair's field row in ring r.
struct RingIt {
    const float *base;
    long long slot_stride, P;
    int S, mod, s, slot;
    __device__ __forceinline__ void init(const RingRef &r, int n0, int S_, long long P_, long long rowoff)
    {
        base = r.base + rowoff; slot_stride = r.slot_stride; P = P_; S = S_; mod = r.mod; s = 0;
        slot = r.mod > 0 ? (n0 + r.shift) % r.mod : r.shift;
    }
    __device__ __forceinline__ const float *ptr() const { return base + (long long)slot * slot_stride + (long long)s * P; }
    __device__ __forceinline__ void next()
    {
        if (++s == S) {
            s = 0;
            if (++slot == mod) slot = 0;   // mod == 0 (direct rings) never wraps
        }
    }
};

// ---- asynchronous global -> shared copies (LDGSTS); src_bytes = 0 zero-fills the 16 bytes
__device__ __forceinline__ void cpa16(float *dst, const float *src, bool valid)
{
    const unsigned d = static_cast<unsigned>(__cvta_generic_to_shared(dst));
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(d), "l"(src), "r"(valid ? 16 : 0) : "memory");
}
__device__ __forceinline__ void cpa_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cpa_wait() { asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory"); }

// Copies the row segment [wal, wal + 4 * nchunk) of `src` (16-byte chunks, zero outside [0, NXP))
// into `dst`; wal is a multiple of 4.
__device__ __forceinline__ void copy_window(float *dst, const float *src, int wal, int nchunk, int NXP)
{
    for (int k = threadIdx.x; k < nchunk; k += EXT_TX) {
        const int col = wal + 4 * k;
        const bool ok = col >= 0 && col + 4 <= NXP;
        cpa16(dst + 4 * k, ok ? src + col : src, ok);
    }
}

// ------------------------------------------------------------------ scatter

// Register-blocked scatter: a thread owns PY outputs y_j = ybase + 2j (j < PY), so the D
// samples they need, y_j - 2 sigma h, fall on the NH + PY - 1 even-spaced positions
// ybase + 2m: one shared-memory load per position serves up to PY multiply-adds.  The
// thread's PY x NH weights stay in registers for the whole segment.  Outputs are staged
// through shared memory and stored coalesced.
// Vector loads from shared memory: VW = 4 (16-byte, LDS.128) or 2 (8-byte, LDS.64) consecutive floats.
template <int VW, int N>
__device__ __forceinline__ void lds_vec(float (&dst)[N], const float *src)
{
    static_assert(N % VW == 0, "window length must be a multiple of the vector width");
    if (VW == 4) {
#pragma unroll
        for (int k = 0; k < N / 4; ++k) {
            const float4 v = reinterpret_cast<const float4 *>(src)[k];
            dst[4 * k] = v.x; dst[4 * k + 1] = v.y; dst[4 * k + 2] = v.z; dst[4 * k + 3] = v.w;
        }
    } else {
#pragma unroll
        for (int k = 0; k < N / 2; ++k) {
            const float2 v = reinterpret_cast<const float2 *>(src)[k];
            dst[2 * k] = v.x; dst[2 * k + 1] = v.y;
        }
    }
}

// Register-blocked scatter: a thread owns PY consecutive outputs y_j = yb + j; the D samples
// they need, y_j - 2 sigma h, lie in the 4 HM + PY consecutive positions [yb - 2HM, yb + PY + 2HM),
// read with conflict-free vector loads (the column range is aligned so that the CTA's window
// starts on a 16-byte boundary).  The PY x NH weights stay in registers for the whole segment.
// The (step, shot) pairs stream through an EXT_STAGES-deep cp.async ring, one barrier per pair.
template <int NH, int PY, int SIGMA>
__global__ void __launch_bounds__(EXT_TX) k_scatter_rb(const ExtArgs a)
{
    extern __shared__ float4 sm4[];
    float *sm = reinterpret_cast<float *>(sm4);
    constexpr int HM = (NH - 1) / 2;
    constexpr int TXS = EXT_TX * PY;               // outputs per CTA
    constexpr int SPAN = TXS + 4 * HM;             // D window, starting at y0 - 2 HM (16-byte aligned)
    constexpr int NCH = (SPAN + 3) / 4;
    constexpr int STG = 4 * NCH + 4;
    constexpr int NS = EXT_STAGES;
    constexpr int NM = PY + 4 * HM;                // samples per thread
    constexpr int VW = (PY % 4 == 0) ? 4 : 2;
    constexpr int NMV = (NM + VW - 1) / VW * VW;
    const int Z = a.z_lo + blockIdx.y;
    const int y0 = a.x_lo + blockIdx.x * TXS;
    const int t = threadIdx.x;
    const int yb = y0 + PY * t;
    const long long rowoff = (long long)Z * a.NXP;
    const int wal = y0 - 2 * HM;                   // multiple of 4 by the launcher's choice of x_lo

    float Wr[PY][NH];
#pragma unroll
    for (int j = 0; j < PY; ++j) {
        const int y = yb + j;
#pragma unroll
        for (int ih = 0; ih < NH; ++ih) {
            const int xs = y - SIGMA * (ih - HM);
            Wr[j][ih] = (y < a.x_hi && xs >= 0 && xs < a.NXP) ? __ldg(a.W + ih * a.P + rowoff + xs) : 0.f;
        }
    }
    RingIt itin, itout;
    itin.init(a.in, a.n0, a.S, a.P, rowoff);
    itout.init(a.outr, a.n0, a.S, a.P, rowoff + yb);
    int stage_in = 0, stage_c = 0;
    auto issue = [&](int p) {
        if (p < a.npair) {
            copy_window(sm + stage_in * STG, itin.ptr(), wal, NCH, a.NXP);
            itin.next();
        }
        stage_in = stage_in + 1 == NS ? 0 : stage_in + 1;
        cpa_commit();
    };
    auto compute = [&](const float *stg, float *o) {
        float dv[NMV];                   // dv[k] = D(yb - 2 HM + k): stage index PY t + k
        lds_vec<VW>(dv, stg + PY * t);
        float acc[PY];
#pragma unroll
        for (int j = 0; j < PY; ++j) acc[j] = 0.f;
#pragma unroll
        for (int ih = 0; ih < NH; ++ih)      // offsets outer: the PY sums are independent chains
#pragma unroll
            for (int j = 0; j < PY; ++j)     // D(y_j - 2 SIGMA h) = dv[j - 2 SIGMA (ih - HM) + 2 HM]
                acc[j] = fmaf(Wr[j][ih], dv[j - 2 * SIGMA * (ih - HM) + 2 * HM], acc[j]);
#pragma unroll
        for (int j = 0; j < PY; j += 2) {
            if (yb + j + 1 < a.x_hi) {
                float2 v = make_float2(acc[j], acc[j + 1]);
                if (a.accumulate) {
                    const float2 old = *reinterpret_cast<const float2 *>(o + j);
                    v.x += old.x; v.y += old.y;
                }
                *reinterpret_cast<float2 *>(o + j) = v;
            } else if (yb + j < a.x_hi) {
                o[j] = a.accumulate ? o[j] + acc[j] : acc[j];
            }
        }
    };
    // two pairs per barrier.  The prologue fills NS - 2 stages; iteration p waits for pairs p and
    // p+1 (at most NS - 4 younger groups pending), then refills the stages of pairs p-2 and p-1,
    // which every thread finished in the previous iteration (the barrier orders it).
#pragma unroll
    for (int q = 0; q < NS - 2; ++q) issue(q);
    for (int p = 0; p < a.npair; p += 2) {
        cpa_wait<NS - 4>();
        __syncthreads();
        issue(p + NS - 2);
        issue(p + NS - 1);
        const float *st0 = sm + stage_c * STG;
        stage_c = stage_c + 1 == NS ? 0 : stage_c + 1;
        const float *st1 = sm + stage_c * STG;
        stage_c = stage_c + 1 == NS ? 0 : stage_c + 1;
        float *o0 = const_cast<float *>(itout.ptr());
        itout.next();
        compute(st0, o0);
        if (p + 1 < a.npair) {
            float *o1 = const_cast<float *>(itout.ptr());
            itout.next();
            compute(st1, o1);
        }
    }
    cpa_wait<0>();
}

// Generic-nh fallback (weights re-read per pair): any odd nh up to MAX_NH.
__global__ void __launch_bounds__(EXT_TX) k_scatter_gen(const ExtArgs a)
{
    extern __shared__ float sm[];
    const int nh = a.nh, hm = (nh - 1) / 2;
    const int Z = a.z_lo + blockIdx.y;
    const int y0 = a.x_lo + blockIdx.x * EXT_TX;
    const int y = y0 + threadIdx.x;
    const bool yin = y < a.x_hi;
    const int span = EXT_TX + 4 * hm;
    const int wbase = y0 - 2 * hm;
    const long long rowoff = (long long)Z * a.NXP;
    float *out_base = const_cast<float *>(a.outr.base);
    for (int p = 0; p < a.npair; ++p) {
        const int j = p / a.S, s = p % a.S, n = a.n0 + j;
        const float *src = a.in.base + ring_off(a.in, n, j) + (long long)s * a.P + rowoff;
        __syncthreads();
        for (int i = threadIdx.x; i < span; i += EXT_TX) {
            const int xp = wbase + i;
            sm[i] = (xp >= 0 && xp < a.NXP) ? __ldg(src + xp) : 0.f;
        }
        __syncthreads();
        float acc = 0.f;
        const int c0 = threadIdx.x + 2 * hm;
        for (int ih = 0; ih < nh; ++ih) {
            const int xs = y - a.sigma * (ih - hm);
            const float wv = (yin && xs >= 0 && xs < a.NXP) ? __ldg(a.W + ih * a.P + rowoff + xs) : 0.f;
            acc = fmaf(wv, sm[c0 - 2 * a.sigma * (ih - hm)], acc);
        }
        if (yin) {
            float *o = out_base + ring_off(a.outr, n, j) + (long long)s * a.P + rowoff + y;
            *o = a.accumulate ? *o + acc : acc;
        }
    }
}

template <int NH, int PY>
static void launch_scatter_nh(const ExtArgs &a, cudaStream_t st)
{
    constexpr int HM = (NH - 1) / 2;
    constexpr int TXS = EXT_TX * PY;
    constexpr int STG = 4 * ((TXS + 4 * HM + 3) / 4) + 4;
    const size_t smem = EXT_STAGES * STG * sizeof(float);
    dim3 grid((a.x_hi - a.x_lo + TXS - 1) / TXS, a.z_hi - a.z_lo);
    static bool attr = false;      // once per instantiation, before any launch (and any capture)
    if (!attr) {
        cudaFuncSetAttribute(k_scatter_rb<NH, PY, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        cudaFuncSetAttribute(k_scatter_rb<NH, PY, -1>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        attr = true;
    }
    if (a.sigma > 0) k_scatter_rb<NH, PY, 1><<<grid, EXT_TX, smem, st>>>(a);
    else k_scatter_rb<NH, PY, -1><<<grid, EXT_TX, smem, st>>>(a);
}

cudaError_t launch_scatter(const ExtArgs &a, cudaStream_t st)
{
    if (a.npair <= 0 || a.x_hi <= a.x_lo || a.z_hi <= a.z_lo) return cudaSuccess;
    switch (a.nh) {
    case 1: launch_scatter_nh<1, 8>(a, st); break;
    case 3: launch_scatter_nh<3, 8>(a, st); break;
    case 5: launch_scatter_nh<5, 8>(a, st); break;
    case 11: launch_scatter_nh<11, 8>(a, st); break;
    case 21: launch_scatter_nh<21, 4>(a, st); break;
    case 31: launch_scatter_nh<31, 2>(a, st); break;
    case 41: launch_scatter_nh<41, 2>(a, st); break;
    default: {
        dim3 grid((a.x_hi - a.x_lo + EXT_TX - 1) / EXT_TX, a.z_hi - a.z_lo);
        const int hm = (a.nh - 1) / 2;
        k_scatter_gen<<<grid, EXT_TX, (EXT_TX + 4 * hm) * sizeof(float), st>>>(a);
    }
    }
    return cudaGetLastError();
}

// ------------------------------------------------------------------ imaging

// Register-blocked imaging: a thread owns PX consecutive points x_i = xb + i and, for
// IMG_EXT, their PX x NH image accumulators (IMG_CONTRACT: PX x NH weights p~ and PX
// accumulators) for the whole segment.  D(x_i - h) and L(x_i + h) come from PX + NH - 1
// window samples each, so a shared-memory load serves up to PX multiply-adds.
template <int NH, int PX, int MODE>
__global__ void __launch_bounds__(EXT_TX) k_image_rb(const ImgArgs a)
{
    extern __shared__ float4 sm4[];
    float *sm = reinterpret_cast<float *>(sm4);
    constexpr int HM = (NH - 1) / 2;
    constexpr int TXS = EXT_TX * PX;
    constexpr int SPAN = TXS + 2 * HM;
    constexpr int NCH = (SPAN + 3) / 4;
    constexpr int WIN = 4 * NCH + 4;
    constexpr int STG = 2 * WIN;                   // D window, then L window
    constexpr int NS = EXT_STAGES;
    constexpr int NW = PX + NH - 1;
    constexpr int VW = (PX % 4 == 0) ? 4 : 2;
    constexpr int NWV = (NW + VW - 1) / VW * VW;
    const int Z = a.z_lo + blockIdx.y;
    const int x0 = a.x_lo + blockIdx.x * TXS;
    const int t = threadIdx.x;
    const int xb = x0 + PX * t;
    const int wal = x0 - HM;                       // multiple of 4 by the launcher's choice of x_lo
    const long long rowoff = (long long)Z * a.NXP;

    constexpr int NA = MODE == IMG_EXT ? PX * NH : PX;
    float acc[NA];
#pragma unroll
    for (int i = 0; i < NA; ++i) acc[i] = 0.f;
    float ptr[MODE == IMG_CONTRACT ? PX * NH : 1];
    if (MODE == IMG_CONTRACT) {
#pragma unroll
        for (int i = 0; i < PX; ++i)
#pragma unroll
            for (int ih = 0; ih < NH; ++ih)
                ptr[i * NH + ih] = (xb + i < a.x_hi) ? __ldg(a.pt + ih * a.P + rowoff + xb + i) : 0.f;
    }
    RingIt itd, itl;
    itd.init(a.D, a.n0, a.S, a.P, rowoff);
    itl.init(a.L, a.n0, a.S, a.P, rowoff);
    int stage_in = 0, stage_c = 0;
    auto issue = [&](int p) {
        if (p < a.npair) {
            float *st = sm + stage_in * STG;
            copy_window(st, itd.ptr(), wal, NCH, a.NXP);
            copy_window(st + WIN, itl.ptr(), wal, NCH, a.NXP);
            itd.next();
            itl.next();
        }
        stage_in = stage_in + 1 == NS ? 0 : stage_in + 1;
        cpa_commit();
    };
    auto compute = [&](const float *stg) {
        // dv[k] = D(xb - HM + k), lv[k] = L(xb - HM + k): stage index PX t + k (conflict-free vector loads)
        const float *bd = stg + PX * t;
        float dv[NWV], lv[NWV];
        lds_vec<VW>(dv, bd);
        lds_vec<VW>(lv, bd + WIN);
#pragma unroll
        for (int i = 0; i < PX; ++i) {
            if (MODE == IMG_EXT) {
#pragma unroll
                for (int ih = 0; ih < NH; ++ih)   // D(x_i - h) = dv[i - ih + 2 HM], L(x_i + h) = lv[i + ih]
                    acc[i * NH + ih] = fmaf(dv[i - ih + 2 * HM], lv[i + ih], acc[i * NH + ih]);
            } else {
                float s = 0.f;
#pragma unroll
                for (int ih = 0; ih < NH; ++ih) s = fmaf(ptr[i * NH + ih] * dv[i - ih + 2 * HM], lv[i + ih], s);
                acc[MODE == IMG_EXT ? 0 : i] += s;
            }
        }
    };
    // two pairs per barrier (same stage accounting as the scatter kernel)
#pragma unroll
    for (int q = 0; q < NS - 2; ++q) issue(q);
    for (int p = 0; p < a.npair; p += 2) {
        cpa_wait<NS - 4>();
        __syncthreads();
        issue(p + NS - 2);
        issue(p + NS - 1);
        const float *st0 = sm + stage_c * STG;
        stage_c = stage_c + 1 == NS ? 0 : stage_c + 1;
        const float *st1 = sm + stage_c * STG;
        stage_c = stage_c + 1 == NS ? 0 : stage_c + 1;
        compute(st0);
        if (p + 1 < a.npair) compute(st1);
    }
    cpa_wait<0>();
#pragma unroll
    for (int i = 0; i < PX; ++i) {
        if (xb + i >= a.x_hi) continue;
        if (MODE == IMG_EXT) {
#pragma unroll
            for (int ih = 0; ih < NH; ++ih) a.img[ih * a.P + rowoff + xb + i] += acc[i * NH + ih];
        } else {
            a.img[rowoff + xb + i] += acc[MODE == IMG_EXT ? 0 : i];
        }
    }
}

// Generic-nh fallback: one point per thread, accumulators in shared memory.
template <int MODE>
__global__ void __launch_bounds__(EXT_TX) k_image_gen(const ImgArgs a)
{
    extern __shared__ float sm[];
    const int nh = a.nh, hm = (nh - 1) / 2;
    const int Z = a.z_lo + blockIdx.y;
    const int x0 = a.x_lo + blockIdx.x * EXT_TX;
    const int X = x0 + threadIdx.x;
    const bool xin = X < a.x_hi;
    const int span = EXT_TX + 2 * hm;
    const int wbase = x0 - hm;
    const long long rowoff = (long long)Z * a.NXP;
    float *bd = sm, *bl = sm + span, *gacc = sm + 2 * span;
    if (MODE == IMG_EXT)
        for (int ih = 0; ih < nh; ++ih) gacc[ih * EXT_TX + threadIdx.x] = 0.f;
    float cacc = 0.f;
    for (int p = 0; p < a.npair; ++p) {
        const int j = p / a.S, s = p % a.S, n = a.n0 + j;
        const float *sd = a.D.base + ring_off(a.D, n, j) + (long long)s * a.P + rowoff;
        const float *sl = a.L.base + ring_off(a.L, n, j) + (long long)s * a.P + rowoff;
        __syncthreads();
        for (int i = threadIdx.x; i < span; i += EXT_TX) {
            const int xp = wbase + i;
            const bool ok = xp >= 0 && xp < a.NXP;
            bd[i] = ok ? __ldg(sd + xp) : 0.f;
            bl[i] = ok ? __ldg(sl + xp) : 0.f;
        }
        __syncthreads();
        const int t = threadIdx.x;
        for (int ih = 0; ih < nh; ++ih) {
            const float prod = bd[t + 2 * hm - ih] * bl[t + ih];
            if (MODE == IMG_EXT) gacc[ih * EXT_TX + t] += prod;
            else cacc = fmaf(xin ? __ldg(a.pt + ih * a.P + rowoff + X) : 0.f, prod, cacc);
        }
    }
    if (!xin) return;
    if (MODE == IMG_EXT)
        for (int ih = 0; ih < nh; ++ih) a.img[ih * a.P + rowoff + X] += gacc[ih * EXT_TX + threadIdx.x];
    else
        a.img[rowoff + X] += cacc;
}

// pointwise (h = 0) accumulation: G += sum_pairs D (alpha L + M2) + Ds L, four independent
// pairs in flight per thread (coalesced: consecutive threads, consecutive points).
__global__ void __launch_bounds__(EXT_TX) k_image_local(const ImgArgs a)
{
    const int Z = a.z_lo + blockIdx.y;
    const int X = a.x_lo + blockIdx.x * EXT_TX + threadIdx.x;
    if (X >= a.x_hi) return;
    const long long off = (long long)Z * a.NXP + X;
    RingIt itd, itl, itm, its;
    itd.init(a.D, a.n0, a.S, a.P, off);
    itl.init(a.L, a.n0, a.S, a.P, off);
    if (a.M2.base) itm.init(a.M2, a.n0, a.S, a.P, off);
    if (a.Ds.base) its.init(a.Ds, a.n0, a.S, a.P, off);
    float acc[4] = {0.f, 0.f, 0.f, 0.f};
    for (int p = 0; p < a.npair; p += 4) {
        // four independent pairs per iteration: their loads are all in flight together
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            if (p + u < a.npair) {
                const float l = __ldg(itl.ptr());
                float tt = a.alpha * l;
                if (a.M2.base) { tt += __ldg(itm.ptr()); itm.next(); }
                float r = __ldg(itd.ptr()) * tt;
                if (a.Ds.base) { r = fmaf(__ldg(its.ptr()), l, r); its.next(); }
                acc[u] += r;
                itd.next();
                itl.next();
            }
        }
    }
    a.img[off] += (acc[0] + acc[1]) + (acc[2] + acc[3]);
}

template <int NH, int PX, int MODE>
static void launch_image_rb(const ImgArgs &a, cudaStream_t st)
{
    constexpr int HM = (NH - 1) / 2;
    constexpr int TXS = EXT_TX * PX;
    constexpr int STG = 2 * (4 * ((TXS + 2 * HM + 3) / 4) + 4);
    const size_t smem = EXT_STAGES * STG * sizeof(float);
    dim3 grid((a.x_hi - a.x_lo + TXS - 1) / TXS, a.z_hi - a.z_lo);
    static bool attr = false;      // once per instantiation, before any launch (and any capture)
    if (!attr) {
        cudaFuncSetAttribute(k_image_rb<NH, PX, MODE>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        attr = true;
    }
    k_image_rb<NH, PX, MODE><<<grid, EXT_TX, smem, st>>>(a);
}

template <int MODE>
static cudaError_t launch_image_mode(const ImgArgs &a, cudaStream_t st)
{
    switch (a.nh) {
    case 1: launch_image_rb<1, 8, MODE>(a, st); break;
    case 3: launch_image_rb<3, 8, MODE>(a, st); break;
    case 5: launch_image_rb<5, 8, MODE>(a, st); break;
    case 11: launch_image_rb<11, 8, MODE>(a, st); break;
    case 21: launch_image_rb<21, 4, MODE>(a, st); break;
    case 31: launch_image_rb<31, 2, MODE>(a, st); break;
    case 41: launch_image_rb<41, 2, MODE>(a, st); break;
    default: {
        const int hm = (a.nh - 1) / 2;
        size_t smem = (2 * (EXT_TX + 2 * hm) + (MODE == IMG_EXT ? a.nh * EXT_TX : 0)) * sizeof(float);
        if (smem > 48 * 1024) {
            cudaError_t e = cudaFuncSetAttribute(k_image_gen<MODE>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                 (int)smem);
            if (e != cudaSuccess) return e;
        }
        dim3 grid((a.x_hi - a.x_lo + EXT_TX - 1) / EXT_TX, a.z_hi - a.z_lo);
        k_image_gen<MODE><<<grid, EXT_TX, smem, st>>>(a);
    }
    }
    return cudaGetLastError();
}

cudaError_t launch_image(const ImgArgs &a, int mode, cudaStream_t st)
{
    if (a.npair <= 0 || a.x_hi <= a.x_lo || a.z_hi <= a.z_lo) return cudaSuccess;
    if (mode == IMG_LOCAL) {
        dim3 grid((a.x_hi - a.x_lo + EXT_TX - 1) / EXT_TX, a.z_hi - a.z_lo);
        k_image_local<<<grid, EXT_TX, 0, st>>>(a);
        return cudaGetLastError();
    }
    if (mode == IMG_EXT) return launch_image_mode<IMG_EXT>(a, st);
    return launch_image_mode<IMG_CONTRACT>(a, st);
}

}  // namespace fwk
