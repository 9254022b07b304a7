// Subsurface-offset extension kernels (Barnier et al., Theory section: Born
// modelling extended with horizontal subsurface offsets, Eq. 1, and its
// adjoint, the extended imaging condition, Eqs. 2-5; tomographic operator,
// Eq. 9).
//
//   scatter    e(y)   = sum_h W(y-h, h) D(y-2h)          (sigma = +1)
//   transpose  z(u)   = sum_h W(u+h, h) L(u+2h)          (sigma = -1)
//   image      I(x,h) += sum_{shots,steps} D(x-h) L(x+h)
//   contract   G(x)   += sum_h p~(x,h) sum D(x-h) L(x+h)  (generic kernel only)
//   local      G(x)   += sum D (alpha L + M2) + Ds L
//
// The weights W = b p~ (nh values per point) are shared by every shot and
// every time step, so these kernels run once per segment of K time steps over
// all K x S (step, shot) pairs of a batch, keeping the weights (scatter) or the
// image accumulators (imaging) in registers for the whole segment, while the
// pairs' rows stream through cp.async rings in shared memory.  Weight and image
// traffic is then 1/(K S) of a per-step formulation.  Both default kernels copy
// rows de-interleaved into their even and odd samples: the products of offset h
// pair samples of one parity (y and y - 2h; x - h and x + h), so a lane that
// owns samples of one parity reuses every loaded sample for several offsets.
#include <algorithm>
#include <utility>

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

// ---- asynchronous global -> shared copies (LDGSTS)
__device__ __forceinline__ void cpa_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cpa_wait() { asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory"); }
// 4-byte asynchronous copy (cp.async.ca); src_bytes = 0 zero-fills.  Used to de-interleave a row
// into its even and odd samples while it is copied into shared memory.
__device__ __forceinline__ void cpa4(unsigned dst, const float *src, bool valid)
{
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;\n" ::"r"(dst), "l"(src), "r"(valid ? 4 : 0) : "memory");
}
// unconditional 4-byte copies dst + C SSTEP <- src + C GSTEP bytes for C in the sequence (immediate
// offsets: one instruction per copy)
template <int SOFF, int GOFF>
__device__ __forceinline__ void cpa4_imm(unsigned dst, const float *src)
{
    asm volatile("cp.async.ca.shared.global [%0+%2], [%1+%3], 4;\n" ::"r"(dst), "l"(src), "n"(SOFF), "n"(GOFF)
                 : "memory");
}
template <int SSTEP, int GSTEP, int... C>
__device__ __forceinline__ void cpa4_run(unsigned dst, const float *src, std::integer_sequence<int, C...>)
{
    (cpa4_imm<SSTEP * C, GSTEP * C>(dst, src), ...);
}

// Row pointer of the (step, shot) pairs of a segment in order (shot fastest), advanced by one
// addition per pair and a multiply only when the time slot changes.
struct PairRow {
    const float *base, *row;
    long long slot_stride, P;
    int S, mod, s, slot;
    // starting at pair p0
    __device__ __forceinline__ void init(const RingRef &r, int n0, int S_, long long P_, long long rowoff, int p0 = 0)
    {
        base = r.base + rowoff; slot_stride = r.slot_stride; P = P_; S = S_; mod = r.mod;
        const int step = p0 / S_;
        s = p0 % S_;
        slot = r.mod > 0 ? (n0 + r.shift + step) % r.mod : r.shift + step;
        row = base + (long long)slot * slot_stride + (long long)s * P_;
    }
    __device__ __forceinline__ void next()
    {
        if (++s == S) {
            s = 0;
            if (++slot == mod) slot = 0;   // mod == 0 (direct rings) never wraps
            row = base + (long long)slot * slot_stride;
        } else {
            row += P;
        }
    }
};

// ------------------------------------------------------------------ scatter

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

// ---------------------------------------------------------- scatter, parity-split (default path)
//
// e(y) = sum_h W(y - sigma h, h) D(y - 2 sigma h) reads D only at samples of y's parity.  A lane
// owns A outputs of one parity, y_j = yf + 2j, whose A x NH products need only A + 2 HM samples of
// that parity: rows are copied into shared memory split into their even and odd samples (4-byte
// cp.async), and every sample a lane loads serves up to A multiply-adds with the A x NH weights it
// keeps in registers for the whole segment.  Lanes 0-15 take the even outputs of the warp's 32 A
// columns, lanes 16-31 the odd ones; one shuffle across the two halves reassembles A consecutive
// outputs per lane for vector stores.  Each warp streams its own window through its own cp.async
// ring, synchronised with __syncwarp only.
#ifndef FWIME_SC_WARPS
#define FWIME_SC_WARPS 4
#endif
#ifndef FWIME_SC_STAGES
#define FWIME_SC_STAGES 8
#endif
#ifndef FWIME_SC_MINB
#define FWIME_SC_MINB 3   // at most 168 registers: 3 CTAs per SM for every nh (nh 31 transposed: 229 -> 168, -3.5 %)
#endif
#ifndef FWIME_IMG_MINB
#define FWIME_IMG_MINB 1
#endif
#ifndef FWIME_SC_A21
#define FWIME_SC_A21 4
#endif
#ifndef FWIME_SC_A31
#define FWIME_SC_A31 4
#endif
// packed two-lane FP32 (f32x2) forms of the multiply-adds, per kernel where they measured faster
// (scatter -1 % at nh 21; imaging -5.5 % at nh 21 (Marmousi2-shaped B~ + B~*), +1.4 % at nh 31
// (North-Sea-shaped gradient), -16 % at nh 41 (Salt-shaped gradient): every nh but 31 packs)
#ifndef FWIME_SC_F32X2
#define FWIME_SC_F32X2 1
#endif
#ifndef FWIME_IMG_F32X2
#define FWIME_IMG_F32X2 1
#endif
#ifndef FWIME_IMG_UNPACKED_NH
#define FWIME_IMG_UNPACKED_NH 31   // the nh whose imaging kernel keeps the scalar form (packed: +1.4 % time)
#endif
#ifndef FWIME_SC_PAIRS
#define FWIME_SC_PAIRS 0      // (step, shot) pairs per loop iteration of the scatter (sharing its weights);
                              // 0: two at nh 21 and 31 (measured -4.3 % at nh 31, -0.6 % at nh 21), else one
#endif
#ifndef FWIME_SC_BALANCE
#define FWIME_SC_BALANCE 1    // split the scatter's pairs over several warps per task to fill the last wave
#endif
#ifndef FWIME_SC_PACK_MAX
#define FWIME_SC_PACK_MAX 96   // largest nh * A whose weights are packed (more spills)
#endif
constexpr int SC_WARPS = FWIME_SC_WARPS;     // warps per CTA (independent pipelines)
constexpr int SC_STAGES = FWIME_SC_STAGES;   // cp.async ring depth per warp

template <int NH, int A>
struct ScatterShape {
    static constexpr int HM = (NH - 1) / 2;
    static constexpr int WOUT = 32 * A;                      // outputs per warp
    static constexpr int SPAN = WOUT + 4 * HM;               // window [yw - 2 HM, yw + WOUT + 2 HM)
    static constexpr int HALF = SPAN / 2;                    // samples of one parity
    static constexpr int OFF = (HALF + 31) / 32 * 32 + 16;   // odd samples, 16 banks after the even ones
    static constexpr int STG = 2 * OFF;                      // floats per stage
    static constexpr int NCP = (SPAN + 31) / 32;             // 4-byte copies per lane and pair
    static constexpr int VW = A % 4 == 0 ? 4 : 2;
    static constexpr int NWIN = A + 2 * HM;                  // samples a lane reads
    static constexpr int NWV = (NWIN + VW - 1) / VW * VW;
    static constexpr size_t SMEM = (size_t)SC_WARPS * SC_STAGES * STG * sizeof(float);
    // copies past SPAN land below OFF (even) or 2 OFF (odd); reads stay below HALF + 4 <= OFF
    static_assert(OFF >= HALF + 16 && 15 * A + NWV <= OFF, "parity array overflow");
};

// SPLIT: each (row, column block) task's pairs are divided among nsplit warps
template <int NH, int A, int SIGMA, bool SPLIT>
__global__ void __launch_bounds__(SC_WARPS * 32, FWIME_SC_MINB) k_scatter_ps(const ExtArgs a, int nwx, int nsplit)
{
    using Sh = ScatterShape<NH, A>;
    constexpr int HM = Sh::HM, NS = SC_STAGES;
    extern __shared__ float4 sm4[];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    float *wsm = reinterpret_cast<float *>(sm4) + warp * NS * Sh::STG;
    // Warps are numbered over (row, column block[, part]) so that no warp of a CTA idles at a row's end;
    // with SPLIT each of a task's nsplit parts takes an equal share of its (step, shot) pairs, the split
    // chosen on the host so that the segment-long CTAs fill their last wave (the unsplit variant keeps
    // the whole range, a kernel parameter, out of its registers).  Warps share nothing: no block-wide
    // barrier follows.
    const int gw = blockIdx.x * SC_WARPS + warp;   // 32-bit indexing (64-bit indexing spilled at nh 31)
    if (gw >= nwx * (a.z_hi - a.z_lo) * (SPLIT ? nsplit : 1)) return;
    const int task = SPLIT ? gw / nsplit : gw;
    int pb = 0, pe = a.npair;
    if constexpr (SPLIT) {
        const int part = (int)(gw % nsplit);
        pb = (int)((long long)part * a.npair / nsplit);
        pe = (int)((long long)(part + 1) * a.npair / nsplit);
        if (pb == pe) return;
    }
    const int Z = a.z_lo + task / nwx;
    const int yw = a.x_lo + (task % nwx) * Sh::WOUT;  // multiple of 4
    const int par = lane >> 4, tp = lane & 15;
    const int yf = yw + par + 2 * A * tp;          // this lane's outputs yf + 2j, j < A
    const long long rowoff = (long long)Z * a.NXP;
    const int wal = yw - 2 * HM;                   // even

    float Wr[A][NH];
#pragma unroll
    for (int j = 0; j < A; ++j) {
        const int y = yf + 2 * j;
#pragma unroll
        for (int ih = 0; ih < NH; ++ih) {
            const int xs = y - SIGMA * (ih - HM);
            Wr[j][ih] = (y < a.x_hi && xs >= 0 && xs < a.NXP) ? __ldg(a.W + ih * a.P + rowoff + xs) : 0.f;
        }
    }
    // packed two-lane arithmetic where the weights leave room for their pairs (no spills)
    constexpr bool PACK = FWIME_SC_F32X2 && NH * A <= FWIME_SC_PACK_MAX;
    // Packed form: output j reads dv[j + o] at offset ih, o = HM - SIGMA (ih - HM), and o has the
    // parity of ih.  For even o the pairs of outputs (0, 1) and (2, 3) read the aligned register
    // pairs (dv[o], dv[o + 1]), (dv[o + 2], dv[o + 3]); for odd o the pair (1, 2) reads the aligned
    // (dv[o + 1], dv[o + 2]) and outputs 0 and 3 stay scalar.  Each output sums its even-o and
    // odd-o products separately (two chains, as in the scalar form).
    constexpr int NE = PACK ? (NH + 1) / 2 : 1, NO = PACK && NH / 2 > 0 ? NH / 2 : 1;   // even / odd o (o = ih mod 2)
    f32x2 WE[NE][A / 2], WO[NO];
    float WO0[NO], WO3[NO];
#pragma unroll
    for (int ih = 0; ih < (PACK ? NH : 0); ++ih) {
        if (ih % 2 == 0) {
#pragma unroll
            for (int q = 0; q < A / 2; ++q) WE[ih / 2][q] = pk(Wr[2 * q][ih], Wr[2 * q + 1][ih]);
        } else if (A == 4) {
            WO[ih / 2] = pk(Wr[1][ih], Wr[A - 2][ih]);
            WO0[ih / 2] = Wr[0][ih];
            WO3[ih / 2] = Wr[A - 1][ih];
        } else {
            WO0[ih / 2] = Wr[0][ih];
            WO3[ih / 2] = Wr[A - 1][ih];
        }
    }
    // the lane copies window samples n = lane + 32 c (column wal + n) into its parity's array
    const unsigned sm0 =
        static_cast<unsigned>(__cvta_generic_to_shared(wsm)) + 4u * ((lane & 1) * Sh::OFF + (lane >> 1));
    const int col0 = wal + lane;
    const bool interior = wal >= 0 && wal + 32 * Sh::NCP <= a.NXP;
    PairRow pin, pout;
    pin.init(a.in, a.n0, a.S, a.P, rowoff, pb);
    pout.init(a.outr, a.n0, a.S, a.P, rowoff, pb);
    unsigned st_in = 0;
    int st_c = 0;
    auto issue = [&](int p) {
        if (p < pe) {
            const unsigned d = sm0 + st_in;
            // samples n = lane + 32 c of the window [0, SPAN): the last round copies only its first REM
            // lanes' samples (nothing past the window is read, from memory or from shared memory)
            constexpr int REM = Sh::SPAN - 32 * (Sh::NCP - 1);
            if (interior) {
                cpa4_run<64, 128>(d, pin.row + col0, std::make_integer_sequence<int, Sh::NCP - 1>{});
                if (REM == 32 || lane < REM) cpa4_imm<64 * (Sh::NCP - 1), 128 * (Sh::NCP - 1)>(d, pin.row + col0);
            } else {
#pragma unroll
                for (int c = 0; c < Sh::NCP; ++c) {
                    if (c == Sh::NCP - 1 && REM < 32 && lane >= REM) break;
                    const int col = col0 + 32 * c;
                    const bool ok = col >= 0 && col < a.NXP;
                    cpa4(d + 64u * c, pin.row + (ok ? col : 0), ok);
                }
            }
            pin.next();
        }
        st_in = st_in + 4u * Sh::STG == 4u * NS * Sh::STG ? 0u : st_in + 4u * Sh::STG;
        cpa_commit();
    };
    // PP pairs per iteration share the weights: PP independent sets of accumulator chains per warp
    constexpr int PP = FWIME_SC_PAIRS > 0 ? FWIME_SC_PAIRS : (NH == 21 || NH == 31 ? 2 : 1);
    static_assert(NS >= 2 * PP, "ring too short for the pairs per iteration");
#pragma unroll 1
    for (int q = 0; q < NS - PP; ++q) issue(pb + q);
    const int ys = yw + 2 * A * tp + A * par;      // first of the A consecutive outputs this lane stores
    const float *lsm = wsm + par * Sh::OFF + A * tp;
#pragma unroll 1
    for (int p = pb; p < pe; p += PP) {
        cpa_wait<NS - 2 * PP>();                   // pairs p .. p + PP - 1 have landed (this lane's copies) ...
        __syncwarp();                              // ... and every lane's; all finished the pairs before
#pragma unroll
        for (int u = 0; u < PP; ++u) issue(p + NS - PP + u);   // refills the stages of the previous pairs
        float dv[PP][Sh::NWV];                     // dv[u][k] = D(yf - 2 HM + 2k) of pair p + u
#pragma unroll
        for (int u = 0; u < PP; ++u) {
            lds_vec<Sh::VW>(dv[u], lsm + st_c);
            st_c = st_c + Sh::STG == NS * Sh::STG ? 0 : st_c + Sh::STG;
        }
        float e[PP][A];
        if constexpr (PACK) {
            f32x2 ae[PP][A / 2], ao[PP];
            float ao0[PP], ao3[PP];
#pragma unroll
            for (int u = 0; u < PP; ++u) {
                ao[u] = pk(0.f, 0.f);
                ao0[u] = ao3[u] = 0.f;
#pragma unroll
                for (int q = 0; q < A / 2; ++q) ae[u][q] = pk(0.f, 0.f);
            }
#pragma unroll
            for (int m = 0; m < NH; ++m) {                 // offsets in the order of their samples
                const int ih = SIGMA > 0 ? NH - 1 - m : m;
                const int o = HM - SIGMA * (ih - HM);
#pragma unroll
                for (int u = 0; u < PP; ++u) {             // the pairs' chains interleaved
                    if (ih % 2 == 0) {
#pragma unroll
                        for (int q = 0; q < A / 2; ++q)
                            ae[u][q] = fma2(WE[ih / 2][q], pk(dv[u][o + 2 * q], dv[u][o + 2 * q + 1]), ae[u][q]);
                    } else {
                        if (A == 4) ao[u] = fma2(WO[ih / 2], pk(dv[u][o + 1], dv[u][o + 2]), ao[u]);
                        ao0[u] = fmaf(WO0[ih / 2], dv[u][o], ao0[u]);
                        ao3[u] = fmaf(WO3[ih / 2], dv[u][o + A - 1], ao3[u]);
                    }
                }
            }
#pragma unroll
            for (int u = 0; u < PP; ++u) {
                float el[A], ol[A];
#pragma unroll
                for (int q = 0; q < A / 2; ++q) upk(ae[u][q], el[2 * q], el[2 * q + 1]);
                ol[0] = ao0[u];
                ol[A - 1] = ao3[u];
                if (A == 4) upk(ao[u], ol[1], ol[A - 2]);
#pragma unroll
                for (int j = 0; j < A; ++j) e[u][j] = el[j] + ol[j];
            }
        } else {
            // two partial sums per output (even / odd offsets): 2 A independent chains per pair.  Offsets
            // are visited in the order of their samples, so the first products wait only for the first load.
            float acc[PP][2][A];
#pragma unroll
            for (int u = 0; u < PP; ++u)
#pragma unroll
                for (int j = 0; j < A; ++j) acc[u][0][j] = acc[u][1][j] = 0.f;
#pragma unroll
            for (int m = 0; m < NH; ++m) {
                const int ih = SIGMA > 0 ? NH - 1 - m : m;
#pragma unroll
                for (int u = 0; u < PP; ++u)
#pragma unroll
                    for (int j = 0; j < A; ++j)            // D(y_j - 2 SIGMA h) = dv[j - SIGMA (ih - HM) + HM]
                        acc[u][m & 1][j] = fmaf(Wr[j][ih], dv[u][j - SIGMA * (ih - HM) + HM], acc[u][m & 1][j]);
            }
#pragma unroll
            for (int u = 0; u < PP; ++u)
#pragma unroll
                for (int j = 0; j < A; ++j) e[u][j] = acc[u][0][j] + acc[u][1][j];
        }
#pragma unroll
        for (int u = 0; u < PP; ++u) {
            if (PP > 1 && p + u >= pe) break;   // warp-uniform
            float v[A];
            if constexpr (A == 4) {
                const float r0 = __shfl_xor_sync(0xffffffffu, par ? e[u][0] : e[u][2], 16);
                const float r1 = __shfl_xor_sync(0xffffffffu, par ? e[u][1] : e[u][3], 16);
                v[0] = par ? r0 : e[u][0]; v[1] = par ? e[u][2] : r0;
                v[2] = par ? r1 : e[u][1]; v[3] = par ? e[u][3] : r1;
            } else {
                const float r0 = __shfl_xor_sync(0xffffffffu, par ? e[u][0] : e[u][1], 16);
                v[0] = par ? r0 : e[u][0]; v[1] = par ? e[u][1] : r0;
            }
            float *o = const_cast<float *>(pout.row) + ys;
            pout.next();
            if (ys + A <= a.x_hi) {
                if constexpr (A == 4) {
                    float4 w4 = make_float4(v[0], v[1], v[2], v[3]);
                    if (a.accumulate) {
                        const float4 old = *reinterpret_cast<const float4 *>(o);
                        w4.x += old.x; w4.y += old.y; w4.z += old.z; w4.w += old.w;
                    }
                    *reinterpret_cast<float4 *>(o) = w4;
                } else {
                    float2 w2 = make_float2(v[0], v[1]);
                    if (a.accumulate) {
                        const float2 old = *reinterpret_cast<const float2 *>(o);
                        w2.x += old.x; w2.y += old.y;
                    }
                    *reinterpret_cast<float2 *>(o) = w2;
                }
            } else {
#pragma unroll
                for (int k = 0; k < A; ++k)
                    if (ys + k < a.x_hi) o[k] = a.accumulate ? o[k] + v[k] : v[k];
            }
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

template <int NH, int A>
static void launch_scatter_ps(ExtArgs a, cudaStream_t st)
{
    using Sh = ScatterShape<NH, A>;
    a.x_lo -= a.x_lo % 4;          // outputs start on a 16-byte boundary (leading columns get zero weights)
    const int nwx = (a.x_hi - a.x_lo + Sh::WOUT - 1) / Sh::WOUT;        // warps per row
    const long long nw = (long long)nwx * (a.z_hi - a.z_lo);
    constexpr bool CAN_SPLIT = FWIME_SC_BALANCE;
    // once per instantiation, before any launch (and any capture); a function-local static is
    // initialised once even when several host threads launch: the attributes, then the CTAs per SM of
    // the least resident variant
    static const int resident = [] {
        int r[4] = {0, 0, 0, 0};
        const auto setup = [](auto kern, int &res) {
            cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)Sh::SMEM);
            cudaOccupancyMaxActiveBlocksPerMultiprocessor(&res, kern, SC_WARPS * 32, Sh::SMEM);
        };
        setup(k_scatter_ps<NH, A, 1, false>, r[0]);
        setup(k_scatter_ps<NH, A, -1, false>, r[1]);
        r[2] = r[3] = r[0];
        if constexpr (CAN_SPLIT) {
            setup(k_scatter_ps<NH, A, 1, true>, r[2]);
            setup(k_scatter_ps<NH, A, -1, true>, r[3]);
        }
        return std::max(1, std::min(std::min(r[0], r[1]), std::min(r[2], r[3])));
    }();
    // Split every task's pairs into nsplit parts, nsplit <= 8 and parts of at least 4 ring depths of
    // pairs, picked to fill the last wave of resident CTAs best (the smallest within 1 %).
    int nsplit = 1;
    if (CAN_SPLIT) {
        int dev = 0, nsm = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
        const double wave = (double)resident * std::max(nsm, 1);
        auto fill = [&](int k) {   // used fraction of the launch's waves of CTAs
            const double w = std::ceil((double)nw * k / SC_WARPS) / wave;
            return w / std::ceil(w);
        };
        double best = fill(1);
        for (int k = 2; k <= 8 && a.npair / k >= 4 * SC_STAGES; ++k)
            if (fill(k) > best + 0.01) { best = fill(k); nsplit = k; }
    }
    dim3 grid((unsigned)((nw * nsplit + SC_WARPS - 1) / SC_WARPS));
    const int nt = SC_WARPS * 32;
    if (nsplit > 1) {
        if constexpr (CAN_SPLIT) {
            if (a.sigma > 0) k_scatter_ps<NH, A, 1, true><<<grid, nt, Sh::SMEM, st>>>(a, nwx, nsplit);
            else k_scatter_ps<NH, A, -1, true><<<grid, nt, Sh::SMEM, st>>>(a, nwx, nsplit);
        }
    } else if (a.sigma > 0) {
        k_scatter_ps<NH, A, 1, false><<<grid, nt, Sh::SMEM, st>>>(a, nwx, 1);
    } else {
        k_scatter_ps<NH, A, -1, false><<<grid, nt, Sh::SMEM, st>>>(a, nwx, 1);
    }
}

cudaError_t launch_scatter(const ExtArgs &a, cudaStream_t st)
{
    if (a.npair <= 0 || a.x_hi <= a.x_lo || a.z_hi <= a.z_lo) return cudaSuccess;
    switch (a.nh) {
    case 1: launch_scatter_ps<1, 4>(a, st); break;
    case 3: launch_scatter_ps<3, 4>(a, st); break;
    case 5: launch_scatter_ps<5, 4>(a, st); break;
    case 11: launch_scatter_ps<11, 4>(a, st); break;
    case 21: launch_scatter_ps<21, FWIME_SC_A21>(a, st); break;
    case 31: launch_scatter_ps<31, FWIME_SC_A31>(a, st); break;
    case 41: launch_scatter_ps<41, 2>(a, st); break;
    default: {
        dim3 grid((a.x_hi - a.x_lo + EXT_TX - 1) / EXT_TX, a.z_hi - a.z_lo);
        const int hm = (a.nh - 1) / 2;
        k_scatter_gen<<<grid, EXT_TX, (EXT_TX + 4 * hm) * sizeof(float), st>>>(a);
    }
    }
    return cudaGetLastError();
}

// ------------------------------------------------------------------ imaging

// ---------------------------------------------------------- imaging, parity-split blocks (default path)
//
// I(x, h) += D(x - h) L(x + h).  With u = x - h and w = x + h (same parity) the products of one
// (step, shot) pair are D(u) L(w) over the band |w - u| <= 2 HM; in the index of one parity,
// u = ub + par + 2 ut and w = ub + par + 2 wt, the band is |wt - ut| <= HM.  A lane owns 8
// consecutive ut and a window of 4 nl consecutive wt starting lo after its first ut (a task may
// have two windows): 8 + 4 nl loaded samples serve up to 32 nl multiply-adds, products outside the
// band being dropped at compile time.  The windows of the NT tasks (one warp each) tile the band
// exactly, so every (x, h) is accumulated by exactly one lane of one CTA (a CTA covers 256
// consecutive u and every offset).  Rows are copied de-interleaved by parity (4-byte cp.async);
// the 16-byte chunks of a parity array are stored alternately in two halves so that the lanes'
// vector loads, 8 floats apart, hit distinct banks, and so do the copies.
struct ImgTask {
    int lo1, nl1, lo2, nl2;        // windows [lo, lo + 4 nl) of wt - (the lane's first ut); nl2 = 0: none
};

__host__ __device__ constexpr int img_ntask(int nh)
{
    return nh <= 5 ? 1 : nh == 11 ? 2 : nh == 21 ? 3 : nh == 31 ? 4 : 5;
}
__host__ __device__ constexpr ImgTask img_task(int nh, int k)
{
    return nh == 1 ? ImgTask{0, 2, 0, 0}
         : nh <= 5 ? ImgTask{-4, 4, 0, 0}
         : nh == 11 ? (k == 0 ? ImgTask{0, 2, 0, 0} : ImgTask{-8, 2, 8, 2})
         : nh == 21 ? (k == 0 ? ImgTask{-16, 4, 0, 0} : k == 1 ? ImgTask{0, 2, 0, 0} : ImgTask{8, 4, 0, 0})
         : nh == 31 ? (k == 0 ? ImgTask{-8, 2, 0, 0} : k == 1 ? ImgTask{0, 2, 0, 0}
                       : k == 2 ? ImgTask{8, 2, 0, 0} : ImgTask{-16, 2, 16, 2})
         : (k == 0 ? ImgTask{-24, 4, 0, 0} : k == 1 ? ImgTask{-8, 2, 0, 0} : k == 2 ? ImgTask{0, 2, 0, 0}
            : k == 3 ? ImgTask{8, 2, 0, 0} : ImgTask{16, 4, 0, 0});
}
// every wt - ut offset the band needs, -HM .. 7 + HM, lies in exactly one window; none overlap
__host__ __device__ constexpr bool img_tasks_tile(int nh)
{
    const int hm = (nh - 1) / 2;
    for (int o = -64; o < 72; ++o) {
        int n = 0;
        for (int k = 0; k < img_ntask(nh); ++k) {
            const ImgTask t = img_task(nh, k);
            n += (o >= t.lo1 && o < t.lo1 + 4 * t.nl1) + (t.nl2 > 0 && o >= t.lo2 && o < t.lo2 + 4 * t.nl2);
        }
        if (n > 1 || (o >= -hm && o <= 7 + hm && n != 1)) return false;
    }
    return true;
}
static_assert(img_tasks_tile(1) && img_tasks_tile(3) && img_tasks_tile(5) && img_tasks_tile(11) &&
              img_tasks_tile(21) && img_tasks_tile(31) && img_tasks_tile(41), "imaging tasks must tile the band");

// the task whose first window holds offset 0 for all 8 of a lane's ut (wt - ut = 0): it owns h = 0
__host__ __device__ constexpr int img_h0_task(int nh)
{
    for (int k = 0; k < img_ntask(nh); ++k) {
        const ImgTask t = img_task(nh, k);
        if (t.lo1 <= 0 && t.lo1 + 4 * t.nl1 > 7) return k;
    }
    return -1;
}
static_assert(img_h0_task(1) >= 0 && img_h0_task(3) >= 0 && img_h0_task(5) >= 0 && img_h0_task(11) >= 0 &&
              img_h0_task(21) >= 0 && img_h0_task(31) >= 0 && img_h0_task(41) >= 0, "h = 0 in one first window");

__host__ __device__ constexpr int img_hc(int len)     // chunk pairs of a parity array (== 2 mod 8: no conflicts)
{
    int h = 2 * ((len + 15) / 16);
    while (h % 8 != 2) ++h;
    return h;
}

template <int NH>
struct ImgShape {
    static constexpr int HM = (NH - 1) / 2;
    static constexpr int NT = img_ntask(NH);
    static constexpr int TX = 32 * NT;
    static constexpr int lo_min()
    {
        int m = 1 << 20;
        for (int k = 0; k < NT; ++k) {
            const ImgTask t = img_task(NH, k);
            m = t.lo1 < m ? t.lo1 : m;
            if (t.nl2 > 0) m = t.lo2 < m ? t.lo2 : m;
        }
        return m;
    }
    static constexpr int hi_max()
    {
        int m = -(1 << 20);
        for (int k = 0; k < NT; ++k) {
            const ImgTask t = img_task(NH, k);
            m = t.lo1 + 4 * t.nl1 > m ? t.lo1 + 4 * t.nl1 : m;
            if (t.nl2 > 0) m = t.lo2 + 4 * t.nl2 > m ? t.lo2 + 4 * t.nl2 : m;
        }
        return m;
    }
    static constexpr int LO = lo_min();
    static constexpr int UT = 128;                           // ut per parity per CTA (16 lanes x 8)
    static constexpr int LD = UT;                            // D samples per parity
    static constexpr int LL = UT - 8 + hi_max() - LO;        // L samples per parity: wt in [LO, UT - 8 + hi)
    static constexpr int HCD = img_hc(LD), HCL = img_hc(LL);
    static constexpr int OFFD = (8 * HCD + 31) / 32 * 32 + 16, OFFL = (8 * HCL + 31) / 32 * 32 + 16;
    static constexpr int REGD = OFFD + 8 * HCD;              // D region (floats); the L region follows
    static constexpr int STG = (REGD + OFFL + 8 * HCL + 3) / 4 * 4;
    // with the local terms two more D-shaped regions follow (second adjoint field, scattered D2t)
    static constexpr int STGL = STG + 2 * REGD;
    static constexpr int NCD = (2 * LD + TX - 1) / TX, NCL = (2 * LL + TX - 1) / TX;
    static constexpr size_t SMEM = (size_t)EXT_STAGES * STG * sizeof(float);
    static constexpr size_t SMEML = (size_t)EXT_STAGES * STGL * sizeof(float);
    static_assert(REGD % 8 == 0 && LO % 4 == 0, "alignment");
};

// one task's share of a pair: products of the lane's 8 D samples with its L window(s).  LOCAL: the task
// that owns h = 0 also sums the local terms D M2 + Ds L at its 8 points (x = u, where it holds D(u) and L(u))
template <int NH, int K, bool LOCAL = false>
struct ImgTaskBody {
    static constexpr ImgTask T = img_task(NH, K);
    static constexpr bool LH0 = LOCAL && K == img_h0_task(NH);
    static constexpr int HM = (NH - 1) / 2;
    static constexpr int W1 = 4 * T.nl1, W2 = T.nl2 > 0 ? 4 * T.nl2 : 1;
    // packed two-lane form: the products of one D sample with the L pair (2 q, 2 q + 1) of a window
    // accumulate in one register pair when both lie in the band; the band's edge entries whose
    // partner lies outside stay scalar
    static constexpr bool PACK = FWIME_IMG_F32X2 && NH != FWIME_IMG_UNPACKED_NH;   // measured slower at nh 31
    static constexpr int P1 = PACK ? W1 / 2 : 1, P2 = PACK && W2 >= 2 ? W2 / 2 : 1;
    float acc1[8][W1], acc2[8][W2];
    f32x2 pac1[8][P1], pac2[8][P2];
    float loc[LH0 ? 8 : 1];

    __device__ __forceinline__ static constexpr bool in1(int i, int j) { return (T.lo1 + j - i) <= HM && (T.lo1 + j - i) >= -HM; }
    __device__ __forceinline__ static constexpr bool in2(int i, int j)
    {
        return T.nl2 > 0 && (T.lo2 + j - i) <= HM && (T.lo2 + j - i) >= -HM;
    }
    // entry (i, j) accumulates in the pair (i, j / 2)
    __device__ __forceinline__ static constexpr bool pk1(int i, int j) { return PACK && in1(i, j & ~1) && in1(i, j | 1); }
    __device__ __forceinline__ static constexpr bool pk2(int i, int j) { return PACK && in2(i, j & ~1) && in2(i, j | 1); }
    __device__ __forceinline__ void zero()
    {
#pragma unroll
        for (int i = 0; i < 8; ++i) {
#pragma unroll
            for (int j = 0; j < W1; ++j) acc1[i][j] = 0.f;
#pragma unroll
            for (int j = 0; j < W2; ++j) acc2[i][j] = 0.f;
#pragma unroll
            for (int q = 0; q < P1; ++q) pac1[i][q] = pk(0.f, 0.f);
#pragma unroll
            for (int q = 0; q < P2; ++q) pac2[i][q] = pk(0.f, 0.f);
        }
#pragma unroll
        for (int i = 0; i < (LH0 ? 8 : 1); ++i) loc[i] = 0.f;
    }
    // loads the lane's L window [8 b + LOW, 8 b + LOW + 4 NL) of wt: chunks c0 + q of the L region
    // (which starts at wt = LO), chunk c at slot (c & 1) hcl + (c >> 1)
    template <int LOW, int NL>
    __device__ __forceinline__ static void load_window(float (&lv)[4 * NL], const float *sl, int b, int hcl)
    {
        constexpr int c0 = (LOW - ImgShape<NH>::LO) / 4;
#pragma unroll
        for (int q = 0; q < NL; ++q) {
            const int c = c0 + q;
            const float4 v = *reinterpret_cast<const float4 *>(sl + 4 * ((c & 1) * hcl + b + (c >> 1)));
            lv[4 * q] = v.x; lv[4 * q + 1] = v.y; lv[4 * q + 2] = v.z; lv[4 * q + 3] = v.w;
        }
    }
    // the lane's 8 samples of a D-shaped region (its ut = 8 b .. 8 b + 7 of its parity)
    __device__ __forceinline__ static void load8(float (&v)[8], const float *sd, int b)
    {
        const float4 d0 = *reinterpret_cast<const float4 *>(sd + 4 * b);
        const float4 d1 = *reinterpret_cast<const float4 *>(sd + 4 * (ImgShape<NH>::HCD + b));
        v[0] = d0.x; v[1] = d0.y; v[2] = d0.z; v[3] = d0.w;
        v[4] = d1.x; v[5] = d1.y; v[6] = d1.z; v[7] = d1.w;
    }
    // sm2, sds: the lane's parity array of the second adjoint field and the scattered D2t (LOCAL only)
    __device__ __forceinline__ void pair(const float *sd, const float *sl, int b, const float *sm2 = nullptr,
                                         const float *sds = nullptr)
    {
        using Sh = ImgShape<NH>;
        float dv[8];
        load8(dv, sd, b);
        float l1[W1];
        load_window<T.lo1, T.nl1>(l1, sl, b, Sh::HCL);
        if constexpr (LH0) {   // x = u_i: D(u_i) = dv[i], L(u_i) = l1[i - lo1]
            float mv[8], sv[8];
            load8(mv, sm2, b);
            load8(sv, sds, b);
#pragma unroll
            for (int i = 0; i < 8; ++i) loc[i] = fmaf(sv[i], l1[i - T.lo1], fmaf(dv[i], mv[i], loc[i]));
        }
#pragma unroll
        for (int i = 0; i < 8; ++i) {
            const f32x2 dd = pk(dv[i], dv[i]);
#pragma unroll
            for (int j = 0; j < W1; ++j) {
                if (pk1(i, j)) {
                    if (!(j & 1)) pac1[i][j / 2] = fma2(dd, pk(l1[j], l1[j + 1]), pac1[i][j / 2]);
                } else if (in1(i, j)) {
                    acc1[i][j] = fmaf(dv[i], l1[j], acc1[i][j]);
                }
            }
        }
        if constexpr (T.nl2 > 0) {
            float l2[W2];
            load_window<T.lo2, (T.nl2 > 0 ? T.nl2 : 1)>(l2, sl, b, Sh::HCL);
#pragma unroll
            for (int i = 0; i < 8; ++i) {
                const f32x2 dd = pk(dv[i], dv[i]);
#pragma unroll
                for (int j = 0; j < W2; ++j) {
                    if (pk2(i, j)) {
                        if (!(j & 1)) pac2[i][j / 2] = fma2(dd, pk(l2[j], l2[j + 1]), pac2[i][j / 2]);
                    } else if (in2(i, j)) {
                        acc2[i][j] = fmaf(dv[i], l2[j], acc2[i][j]);
                    }
                }
            }
        }
    }
    __device__ __forceinline__ float val1(int i, int j) const
    {
        if (pk1(i, j)) {
            float lo, hi;
            upk(pac1[i][(j / 2) % P1], lo, hi);
            return (j & 1) ? hi : lo;
        }
        return acc1[i][j];
    }
    __device__ __forceinline__ float val2(int i, int j) const
    {
        if (pk2(i, j)) {
            float lo, hi;
            upk(pac2[i][(j / 2) % P2], lo, hi);
            return (j & 1) ? hi : lo;
        }
        return acc2[i][j];
    }
    // adds the accumulators into img at x = x1 + i + o, h = o - i (o = lo + j), x1 = the lane's
    // first u + its first ut offset; only physical columns [x_lo, x_hi).  LOCAL: img_local at x = x1 + 2 i
    // gains alpha x (its h = 0 sum of D L) + its local terms
    __device__ __forceinline__ void store(const ImgArgs &a, long long rowoff, int x1)
    {
        if constexpr (LH0) {
#pragma unroll
            for (int i = 0; i < 8; ++i) {
                const int x = x1 + 2 * i;
                if (x >= a.x_lo && x < a.x_hi)
                    a.img_local[rowoff + x] += fmaf(a.alpha, val1(i, i - T.lo1), loc[i]);
            }
        }
#pragma unroll
        for (int i = 0; i < 8; ++i) {
#pragma unroll
            for (int j = 0; j < W1; ++j) {
                if (in1(i, j)) {
                    const int x = x1 + i + T.lo1 + j;
                    if (x >= a.x_lo && x < a.x_hi) a.img[(T.lo1 + j - i + HM) * a.P + rowoff + x] += val1(i, j);
                }
            }
#pragma unroll
            for (int j = 0; j < W2; ++j) {
                if (in2(i, j)) {
                    const int x = x1 + i + T.lo2 + j;
                    if (x >= a.x_lo && x < a.x_hi) a.img[(T.lo2 + j - i + HM) * a.P + rowoff + x] += val2(i, j);
                }
            }
        }
    }
};

// block-wide barrier that warps may reach from different code (each warp runs its own task's
// instantiation of the same pipeline): the non-.aligned form of bar.sync
__device__ __forceinline__ void cta_barrier() { asm volatile("barrier.sync 0;\n" ::: "memory"); }

template <int NH, int K, bool LOCAL = false>
__device__ __forceinline__ void img_task_run(const ImgArgs &a, int u_lo, float *sm, int lane)
{
    using Sh = ImgShape<NH>;
    constexpr int NS = EXT_STAGES;
    constexpr int STG = LOCAL ? Sh::STGL : Sh::STG;   // floats per stage
    constexpr unsigned MOFF = 4u * Sh::STG, SOFF = 4u * (Sh::STG + Sh::REGD);   // bytes to the local regions
    const int Z = a.z_lo + blockIdx.y;
    const long long rowoff = (long long)Z * a.NXP;
    const int ub = u_lo + 256 * blockIdx.x;         // even
    const int t = threadIdx.x;
    const int par = lane >> 4, b = lane & 15;
    // copy plan: thread t copies window samples n = t + TX c; sample n of a window goes to parity n & 1,
    // index k = n >> 1, chunk k >> 2 stored at slot (chunk & 1) HC + (chunk >> 1)
    const int cw = (t & 1), ch = (t >> 3) & 1, cp = (t >> 4), ce = (t >> 1) & 3;
    const unsigned sbase = static_cast<unsigned>(__cvta_generic_to_shared(sm));
    const unsigned dD = sbase + 4u * (cw * Sh::OFFD + 4 * (ch * Sh::HCD + cp) + ce);
    const unsigned dL = sbase + 4u * (Sh::REGD + cw * Sh::OFFL + 4 * (ch * Sh::HCL + cp) + ce);
    constexpr unsigned CSTEP = 4u * 8u * Sh::NT;     // bytes between copies c and c + 1 (TX / 16 chunk pairs)
    const int colD = ub + t, colL = ub + 2 * Sh::LO + t;
    // all copied columns, [ub + 2 LO, ub + 2 LO + 2 LL) (which contains the D window), inside the row
    const bool interior = ub + 2 * Sh::LO >= 0 && ub + 2 * Sh::LO + 2 * Sh::LL <= a.NXP;
    PairRow pd, pl, pm, ps;
    pd.init(a.D, a.n0, a.S, a.P, rowoff);
    pl.init(a.L, a.n0, a.S, a.P, rowoff);
    if constexpr (LOCAL) {
        pm.init(a.M2, a.n0, a.S, a.P, rowoff);
        ps.init(a.Ds, a.n0, a.S, a.P, rowoff);
    }
    int st_in = 0, st_c = 0;
    constexpr int FD = 2 * Sh::LD / Sh::TX, RD = 2 * Sh::LD - FD * Sh::TX;   // full copy rounds, remainder
    constexpr int FL = 2 * Sh::LL / Sh::TX, RL = 2 * Sh::LL - FL * Sh::TX;
    auto issue = [&](int p) {
        if (p < a.npair) {
            const unsigned so = 4u * st_in * STG;
            if (interior) {
                const float *sd = pd.row + colD, *sl = pl.row + colL;
                cpa4_run<CSTEP, 4 * Sh::TX>(dD + so, sd, std::make_integer_sequence<int, FD>{});
                if (RD > 0 && t < RD) cpa4_imm<CSTEP * FD, 4 * Sh::TX * FD>(dD + so, sd);
                cpa4_run<CSTEP, 4 * Sh::TX>(dL + so, sl, std::make_integer_sequence<int, FL>{});
                if (RL > 0 && t < RL) cpa4_imm<CSTEP * FL, 4 * Sh::TX * FL>(dL + so, sl);
                if constexpr (LOCAL) {   // the second adjoint field and the scattered D2t: D's window and layout
                    const float *smv = pm.row + colD, *ssv = ps.row + colD;
                    cpa4_run<CSTEP, 4 * Sh::TX>(dD + so + MOFF, smv, std::make_integer_sequence<int, FD>{});
                    if (RD > 0 && t < RD) cpa4_imm<CSTEP * FD, 4 * Sh::TX * FD>(dD + so + MOFF, smv);
                    cpa4_run<CSTEP, 4 * Sh::TX>(dD + so + SOFF, ssv, std::make_integer_sequence<int, FD>{});
                    if (RD > 0 && t < RD) cpa4_imm<CSTEP * FD, 4 * Sh::TX * FD>(dD + so + SOFF, ssv);
                }
            } else {
#pragma unroll
                for (int c = 0; c < Sh::NCD; ++c) {
                    if (t + Sh::TX * c < 2 * Sh::LD) {
                        const int col = colD + Sh::TX * c;
                        const bool ok = col >= 0 && col < a.NXP;
                        cpa4(dD + so + CSTEP * c, pd.row + (ok ? col : 0), ok);
                        if constexpr (LOCAL) {
                            cpa4(dD + so + MOFF + CSTEP * c, pm.row + (ok ? col : 0), ok);
                            cpa4(dD + so + SOFF + CSTEP * c, ps.row + (ok ? col : 0), ok);
                        }
                    }
                }
#pragma unroll
                for (int c = 0; c < Sh::NCL; ++c) {
                    if (t + Sh::TX * c < 2 * Sh::LL) {
                        const int col = colL + Sh::TX * c;
                        const bool ok = col >= 0 && col < a.NXP;
                        cpa4(dL + so + CSTEP * c, pl.row + (ok ? col : 0), ok);
                    }
                }
            }
            pd.next();
            pl.next();
            if constexpr (LOCAL) {
                pm.next();
                ps.next();
            }
        }
        st_in = st_in + 1 == NS ? 0 : st_in + 1;
        cpa_commit();
    };
    ImgTaskBody<NH, K, LOCAL> body;
    body.zero();
    // two pairs per barrier: the prologue fills NS - 2 stages; iteration p waits for pairs p and p + 1,
    // then refills the stages of pairs p - 2 and p - 1, which every warp finished before the barrier
#pragma unroll 1
    for (int q = 0; q < NS - 2; ++q) issue(q);
    for (int p = 0; p < a.npair; p += 2) {
        cpa_wait<NS - 4>();
        cta_barrier();
        issue(p + NS - 2);
        issue(p + NS - 1);
        const float *s0 = sm + st_c * STG;
        st_c = st_c + 1 == NS ? 0 : st_c + 1;
        const float *s1 = sm + st_c * STG;
        st_c = st_c + 1 == NS ? 0 : st_c + 1;
        const int pd0 = par * Sh::OFFD;
        body.pair(s0 + pd0, s0 + Sh::REGD + par * Sh::OFFL, b, s0 + Sh::STG + pd0, s0 + Sh::STG + Sh::REGD + pd0);
        if (p + 1 < a.npair)
            body.pair(s1 + pd0, s1 + Sh::REGD + par * Sh::OFFL, b, s1 + Sh::STG + pd0, s1 + Sh::STG + Sh::REGD + pd0);
    }
    cpa_wait<0>();
    // u of the lane's first sample: ub + par + 16 b; x = (u + w) / 2 = ub + par + 16 b + i + o
    body.store(a, rowoff, ub + par + 16 * b);
}

// LOCAL: also the local imaging terms (alpha D L + D M2 + Ds L at h = 0) into img_local, which otherwise
// take their own k_image_local launch re-reading D and L
template <int NH, bool LOCAL = false>
__global__ void __launch_bounds__(ImgShape<NH>::TX, FWIME_IMG_MINB) k_image_ps(const ImgArgs a, int u_lo)
{
    extern __shared__ float4 sm4[];
    float *sm = reinterpret_cast<float *>(sm4);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    constexpr int NT = ImgShape<NH>::NT;
    // warp-uniform dispatch: every warp runs the same pipeline (barriers included) with its own task
    if (warp == 0) img_task_run<NH, 0, LOCAL>(a, u_lo, sm, lane);
    if constexpr (NT > 1) if (warp == 1) img_task_run<NH, 1 % NT, LOCAL>(a, u_lo, sm, lane);
    if constexpr (NT > 2) if (warp == 2) img_task_run<NH, 2 % NT, LOCAL>(a, u_lo, sm, lane);
    if constexpr (NT > 3) if (warp == 3) img_task_run<NH, 3 % NT, LOCAL>(a, u_lo, sm, lane);
    if constexpr (NT > 4) if (warp == 4) img_task_run<NH, 4 % NT, LOCAL>(a, u_lo, sm, lane);
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
// Local imaging: a thread owns 4 consecutive columns (16-byte loads) of one row, a CTA 512 columns, so
// every (step, shot) pair is read as long contiguous row segments; columns start at x_lo rounded down to
// a multiple of 4 and only [x_lo, x_hi) is accumulated.
constexpr int LOC_TX = 128;
__device__ __forceinline__ float4 ldg4e(const float *p) { return __ldg(reinterpret_cast<const float4 *>(p)); }
__global__ void __launch_bounds__(LOC_TX) k_image_local(const ImgArgs a, int xa)
{
    const int Z = a.z_lo + blockIdx.y;
    const int X = xa + 4 * (blockIdx.x * LOC_TX + threadIdx.x);
    if (X >= a.x_hi) return;
    const long long off = (long long)Z * a.NXP + X;
    RingIt itd, itl, itm, its;
    itd.init(a.D, a.n0, a.S, a.P, off);
    itl.init(a.L, a.n0, a.S, a.P, off);
    if (a.M2.base) itm.init(a.M2, a.n0, a.S, a.P, off);
    if (a.Ds.base) its.init(a.Ds, a.n0, a.S, a.P, off);
    float acc[4][4] = {};
    for (int p = 0; p < a.npair; p += 4) {
        // four independent pairs per iteration: their loads are all in flight together
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            if (p + u < a.npair) {
                const float4 l = ldg4e(itl.ptr());
                const float4 d = ldg4e(itd.ptr());
                float4 m2 = make_float4(0.f, 0.f, 0.f, 0.f), ds = m2;
                if (a.M2.base) { m2 = ldg4e(itm.ptr()); itm.next(); }
                if (a.Ds.base) { ds = ldg4e(its.ptr()); its.next(); }
                const float lv[4] = {l.x, l.y, l.z, l.w}, dv[4] = {d.x, d.y, d.z, d.w};
                const float mv[4] = {m2.x, m2.y, m2.z, m2.w}, sv[4] = {ds.x, ds.y, ds.z, ds.w};
#pragma unroll
                for (int c = 0; c < 4; ++c) {
                    float tt = a.alpha * lv[c];
                    if (a.M2.base) tt += mv[c];
                    float r = dv[c] * tt;
                    if (a.Ds.base) r = fmaf(sv[c], lv[c], r);
                    acc[c][u] += r;
                }
                itd.next();
                itl.next();
            }
        }
    }
#pragma unroll
    for (int c = 0; c < 4; ++c)
        if (X + c >= a.x_lo && X + c < a.x_hi) a.img[off + c] += (acc[c][0] + acc[c][1]) + (acc[c][2] + acc[c][3]);
}

template <int MODE>
static cudaError_t launch_image_gen(const ImgArgs &a, cudaStream_t st)
{
    const int hm = (a.nh - 1) / 2;
    size_t smem = (2 * (EXT_TX + 2 * hm) + (MODE == IMG_EXT ? a.nh * EXT_TX : 0)) * sizeof(float);
    if (smem > 48 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(k_image_gen<MODE>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
    }
    dim3 grid((a.x_hi - a.x_lo + EXT_TX - 1) / EXT_TX, a.z_hi - a.z_lo);
    k_image_gen<MODE><<<grid, EXT_TX, smem, st>>>(a);
    return cudaGetLastError();
}

template <int NH>
static void launch_image_ps(const ImgArgs &a, cudaStream_t st)
{
    using Sh = ImgShape<NH>;
    int u_lo = a.x_lo - Sh::HM;    // first u = x - h of the physical columns, made even
    u_lo -= ((u_lo % 2) + 2) % 2;
    dim3 grid((a.x_hi + Sh::HM - u_lo + 255) / 256, a.z_hi - a.z_lo);
    // once per instantiation, before any launch (and any capture), thread-safe (function-local static)
    static const cudaError_t attr =
        cudaFuncSetAttribute(k_image_ps<NH, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)Sh::SMEM) ==
                cudaSuccess
            ? cudaFuncSetAttribute(k_image_ps<NH, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)Sh::SMEML)
            : cudaErrorUnknown;
    (void)attr;
    if (a.img_local) k_image_ps<NH, true><<<grid, Sh::TX, Sh::SMEML, st>>>(a, u_lo);
    else k_image_ps<NH, false><<<grid, Sh::TX, Sh::SMEM, st>>>(a, u_lo);
}

template <int MODE>
static cudaError_t launch_image_mode(const ImgArgs &a, cudaStream_t st)
{
    if (MODE != IMG_EXT) return launch_image_gen<MODE>(a, st);
    if (a.img_local && (a.nh != 1 && a.nh != 3 && a.nh != 5 && a.nh != 11 && a.nh != 21 && a.nh != 31 && a.nh != 41)) {
        // generic nh: the extended image, then the local terms in their own kernel
        ImgArgs e = a;
        e.img_local = nullptr;
        const cudaError_t err = launch_image_gen<MODE>(e, st);
        if (err != cudaSuccess) return err;
        ImgArgs l = a;
        l.img = a.img_local;
        l.img_local = nullptr;
        return launch_image(l, IMG_LOCAL, st);
    }
    switch (a.nh) {
    case 1: launch_image_ps<1>(a, st); break;
    case 3: launch_image_ps<3>(a, st); break;
    case 5: launch_image_ps<5>(a, st); break;
    case 11: launch_image_ps<11>(a, st); break;
    case 21: launch_image_ps<21>(a, st); break;
    case 31: launch_image_ps<31>(a, st); break;
    case 41: launch_image_ps<41>(a, st); break;
    default: return launch_image_gen<MODE>(a, st);
    }
    return cudaGetLastError();
}

cudaError_t launch_image(const ImgArgs &a, int mode, cudaStream_t st)
{
    if (a.npair <= 0 || a.x_hi <= a.x_lo || a.z_hi <= a.z_lo) return cudaSuccess;
    if (mode == IMG_LOCAL) {
        const int xa = a.x_lo - a.x_lo % 4;   // 16-byte aligned: rows are NXP (a multiple of 32) floats apart
        dim3 grid((a.x_hi - xa + 4 * LOC_TX - 1) / (4 * LOC_TX), a.z_hi - a.z_lo);
        k_image_local<<<grid, LOC_TX, 0, st>>>(a, xa);
        return cudaGetLastError();
    }
    if (mode == IMG_EXT) return launch_image_mode<IMG_EXT>(a, st);
    return launch_image_mode<IMG_CONTRACT>(a, st);
}

}  // namespace fwk
