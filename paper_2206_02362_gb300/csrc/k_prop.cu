// One time step of the 2-D acoustic constant-density wave equation, 2nd order
// in time and 8th order in space, with the Cerjan-type sponge fused in
// (Barnier et al., Theory section: the acoustic isotropic constant-density
// two-way operator f of Eq. 1; Marmousi2 section: absorbing boundaries on all
// sides):
//
//   q^{n+1} = g (2 q^n - g q^{n-1} + c (L q^n + s^n)),   g = gz[IZ] gx[IX],  c = v^2 dt^2
//
// The same kernel advances the adjoint wavefield backward in time: with
// mu = c g lambda the exact transpose of the recursion takes the same form
// (mu^n from mu^{n+1}, mu^{n+2}), so forward and adjoint share this code.
//
// Work decomposition (HBM-bound, no tensor cores): one warp owns a strip of
// 128 x-points (32 lanes x float4) and a chunk of rows, marching down z with a
// 9-row register queue, so every row of q^n is read from memory once per
// strip; the +-4 x-neighbours come from the adjacent lanes by warp shuffles
// and, at the strip edges, one extra float4 per row.  q^{n-1}, c and the
// output are touched once, coalesced.  Sources (point, dense local terms) and
// the second time derivative (for Born-type scattering) are fused in.
#include "fwime_kernels.cuh"

namespace fwk {

__device__ __forceinline__ float4 f4zero() { return make_float4(0.f, 0.f, 0.f, 0.f); }
__device__ __forceinline__ float4 ldg4(const float *p) { return __ldg(reinterpret_cast<const float4 *>(p)); }
__device__ __forceinline__ float4 ld4(const float *p) { return *reinterpret_cast<const float4 *>(p); }
__device__ __forceinline__ void st4(float *p, float4 v) { *reinterpret_cast<float4 *>(p) = v; }
__device__ __forceinline__ float cmp(const float4 &v, int j)
{
    return j == 0 ? v.x : (j == 1 ? v.y : (j == 2 ? v.z : v.w));
}
__device__ __forceinline__ float4 shfl_up4(float4 v)
{
    v.x = __shfl_up_sync(0xffffffffu, v.x, 1);
    v.y = __shfl_up_sync(0xffffffffu, v.y, 1);
    v.z = __shfl_up_sync(0xffffffffu, v.z, 1);
    v.w = __shfl_up_sync(0xffffffffu, v.w, 1);
    return v;
}
__device__ __forceinline__ float4 shfl_down4(float4 v)
{
    v.x = __shfl_down_sync(0xffffffffu, v.x, 1);
    v.y = __shfl_down_sync(0xffffffffu, v.y, 1);
    v.z = __shfl_down_sync(0xffffffffu, v.z, 1);
    v.w = __shfl_down_sync(0xffffffffu, v.w, 1);
    return v;
}

// ---- asynchronous global -> shared copies (LDGSTS); src_bytes = 0 zero-fills the 16 bytes
__device__ __forceinline__ void cp16(float *dst, const float *src, bool valid)
{
    const unsigned d = static_cast<unsigned>(__cvta_generic_to_shared(dst));
    const int n = valid ? 16 : 0;
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(d), "l"(src), "r"(n) : "memory");
}
// the same copy issued only where `pred` holds (a predicated instruction instead of a divergent branch)
__device__ __forceinline__ void cp16p(float *dst, const float *src, bool valid, bool pred)
{
    const unsigned d = static_cast<unsigned>(__cvta_generic_to_shared(dst));
    const int n = valid ? 16 : 0;
    asm volatile("{\n .reg .pred p;\n setp.ne.b32 p, %3, 0;\n @p cp.async.cg.shared.global [%0], [%1], 16, %2;\n}\n" ::"r"(d),
                 "l"(src), "r"(n), "r"((int)pred)
                 : "memory");
}
__device__ __forceinline__ void cp_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_wait() { asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory"); }
__device__ __forceinline__ float4 lds4(const float *p) { return *reinterpret_cast<const float4 *>(p); }

// Per-warp pipeline: an 8-slot ring of q^n rows (128 points + 4-point halos) feeds the x-taps
// and the register queue; a 4-slot ring holds the q^{n-1}, c and local-source rows of the
// output row.  Iteration z waits for the copy group issued 4 iterations earlier, so about four
// rows of every input stream are in flight per warp.
#ifndef FWIME_PROP_CUR_SLOTS
#define FWIME_PROP_CUR_SLOTS 8
#endif
#ifndef FWIME_PROP_AUX_SLOTS
#define FWIME_PROP_AUX_SLOTS 4
#endif
// Variants k_prop<LOC, D2, SRC>: LOC = 0 no dense local source, 1 exactly one (f0, weight a0), 2 the
// general sum a0 f0 + a1 f1 + a2 f2 + coef fc; D2 writes D2t; SRC adds the point source.  Register
// bounds (minimum resident CTAs) per kind:
#ifndef FWIME_PROP_MIN_BLOCKS
#define FWIME_PROP_MIN_BLOCKS 1   // general local sources (up to five extra rows per stage)
#endif
#ifndef FWIME_PROP_PRED
#define FWIME_PROP_PRED 1   // halo copies predicated, not branched (-0.5 %)
#endif
#ifndef FWIME_PROP_MINB_LOC1
#define FWIME_PROP_MINB_LOC1 3   // one local source: up to 128 registers, 4 CTAs per SM like the plain variants
#endif
#ifndef FWIME_PROP_MINB_PLAIN
#define FWIME_PROP_MINB_PLAIN 3   // up to 128 registers: still 4 CTAs per SM, fewer rematerialised operands
#endif
constexpr int CUR_SLOTS = FWIME_PROP_CUR_SLOTS;   // q^n rows in flight: the queue reads row z+4 of slots
constexpr int AUX_SLOTS = FWIME_PROP_AUX_SLOTS;   // pipeline depth of the q^{n-1}, c, local-source rows
constexpr int CUR_ROW = STRIP + 8;
static_assert(CUR_SLOTS >= AUX_SLOTS + 4, "the q^n ring must hold rows z .. z+4+depth");

// The arithmetic of one output row of a lane (four consecutive columns): the Laplacian from the
// x-neighbours (L | Q4 | Rr, 12 consecutive samples) and the nine queue rows Q0..Q8 (the output row
// is Q4), then the sponge-damped update and optionally D2t.  In the scalar form every product and
// sum is the same as
//   lap = (ax0 + az0) q + sum_k ax_k (q[x-k] + q[x+k]) + sum_k az_k (q[z-k] + q[z+k])   (k = 1..4)
//   out = g (2 q - g p + c (lap + s)),   d2 = (out - 2 q + p) / dt^2.
#ifndef FWIME_PROP_F32X2
#define FWIME_PROP_F32X2 1
#endif
#ifndef FWIME_PROP_F32X2_PLAIN
#define FWIME_PROP_F32X2_PLAIN 1
#endif
// Packed two-lane FP32 (f32x2, see fwime_kernels.cuh) on columns (j, j + 1): half the floating-point
// issue slots of the scalar form, with its rounding.  The coefficient operands as register pairs:
struct PropK {
    f32x2 axc, kx[5], kz[5], inv, a0, a1, a2;
};
__device__ __forceinline__ PropK prop_k(const PropArgs &a)
{
    PropK K;
    K.axc = bits(a.axc2);
#pragma unroll
    for (int k = 1; k < 5; ++k) {
        K.kx[k] = bits(a.kx2[k]);
        K.kz[k] = bits(a.kz2[k]);
    }
    K.inv = bits(a.inv2);
    K.a0 = bits(a.a02);
    K.a1 = bits(a.a12);
    K.a2 = bits(a.a22);
    return K;
}
// columns (2 h, 2 h + 1) of a float4
__device__ __forceinline__ f32x2 half2(const float4 &v, int h) { return h == 0 ? pk(v.x, v.y) : pk(v.z, v.w); }

template <int LOC, bool D2, bool SRC>
__device__ __forceinline__ void row_math_pk(const PropArgs &a, const PropK &K, const float4 &L, const float4 &Q0, const float4 &Q1,
                                         const float4 &Q2, const float4 &Q3, const float4 &Q4, const float4 &Q5,
                                         const float4 &Q6, const float4 &Q7, const float4 &Q8, const float4 &Rr,
                                         const float4 &pv, const float4 &cv, const float4 &lf0, const float4 &lf1,
                                         const float4 &lf2, const float4 &lcf, const float4 &lfc, float gzz,
                                         const float4 &gxv, int sj, float amp, float4 &o, float4 &d2)
{
    constexpr bool LOCAL = LOC > 0;
    const float rr[12] = {L.x, L.y, L.z, L.w, Q4.x, Q4.y, Q4.z, Q4.w, Rr.x, Rr.y, Rr.z, Rr.w};
    const f32x2 GZ = pk(gzz, gzz), NGZ = pk(-gzz, -gzz);
    float ov[4], dv[4];
#pragma unroll
    for (int h = 0; h < 2; ++h) {
        const int j = 2 * h;
        const f32x2 C0 = half2(Q4, h);
        f32x2 lap = mul2(K.axc, C0);
        lap = fma2(K.kx[1], add2(pk(rr[j + 3], rr[j + 4]), pk(rr[j + 5], rr[j + 6])), lap);
        lap = fma2(K.kx[2], add2(pk(rr[j + 2], rr[j + 3]), pk(rr[j + 6], rr[j + 7])), lap);
        lap = fma2(K.kx[3], add2(pk(rr[j + 1], rr[j + 2]), pk(rr[j + 7], rr[j + 8])), lap);
        lap = fma2(K.kx[4], add2(pk(rr[j + 0], rr[j + 1]), pk(rr[j + 8], rr[j + 9])), lap);
        lap = fma2(K.kz[1], add2(half2(Q3, h), half2(Q5, h)), lap);
        lap = fma2(K.kz[2], add2(half2(Q2, h), half2(Q6, h)), lap);
        lap = fma2(K.kz[3], add2(half2(Q1, h), half2(Q7, h)), lap);
        lap = fma2(K.kz[4], add2(half2(Q0, h), half2(Q8, h)), lap);
        if (LOCAL || SRC) {
            f32x2 sv = pk(0.f, 0.f);
            if (LOCAL) {
                sv = fma2(K.a0, half2(lf0, h), sv);
                if (LOC == 2) {
                    sv = fma2(K.a1, half2(lf1, h), sv);
                    sv = fma2(K.a2, half2(lf2, h), sv);
                    sv = fma2(half2(lcf, h), half2(lfc, h), sv);
                }
            }
            if (SRC) sv = add2(sv, pk(sj == j ? amp : 0.f, sj == j + 1 ? amp : 0.f));
            lap = add2(lap, sv);
        }
        const f32x2 GX = half2(gxv, h);
        const f32x2 G = mul2(GZ, GX), NG = mul2(NGZ, GX);
        const f32x2 P = half2(pv, h);
        const f32x2 TC = add2(C0, C0);
        const f32x2 O = mul2(G, fma2(half2(cv, h), lap, fma2(NG, P, TC)));
        upk(O, ov[j], ov[j + 1]);
        if (D2) {
            const f32x2 D = mul2(add2(sub2(O, TC), P), K.inv);
            upk(D, dv[j], dv[j + 1]);
        }
    }
    o = make_float4(ov[0], ov[1], ov[2], ov[3]);
    if (D2) d2 = make_float4(dv[0], dv[1], dv[2], dv[3]);
}
template <int LOC, bool D2, bool SRC>
__device__ __forceinline__ void row_math_sc(const PropArgs &a, const float4 &L, const float4 &Q0, const float4 &Q1,
                                         const float4 &Q2, const float4 &Q3, const float4 &Q4, const float4 &Q5,
                                         const float4 &Q6, const float4 &Q7, const float4 &Q8, const float4 &Rr,
                                         const float4 &pv, const float4 &cv, const float4 &lf0, const float4 &lf1,
                                         const float4 &lf2, const float4 &lcf, const float4 &lfc, float gzz,
                                         const float4 &gxv, int sj, float amp, float4 &o, float4 &d2)
{
    constexpr bool LOCAL = LOC > 0;
    const float rr[12] = {L.x, L.y, L.z, L.w, Q4.x, Q4.y, Q4.z, Q4.w, Rr.x, Rr.y, Rr.z, Rr.w};
    const float axc = a.ax[0] + a.az[0];
    float ov[4], dv[4];
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        const float c0v = rr[j + 4];
        float lap = axc * c0v;
        lap = fmaf(a.ax[1], rr[j + 3] + rr[j + 5], lap);
        lap = fmaf(a.ax[2], rr[j + 2] + rr[j + 6], lap);
        lap = fmaf(a.ax[3], rr[j + 1] + rr[j + 7], lap);
        lap = fmaf(a.ax[4], rr[j + 0] + rr[j + 8], lap);
        lap = fmaf(a.az[1], cmp(Q3, j) + cmp(Q5, j), lap);
        lap = fmaf(a.az[2], cmp(Q2, j) + cmp(Q6, j), lap);
        lap = fmaf(a.az[3], cmp(Q1, j) + cmp(Q7, j), lap);
        lap = fmaf(a.az[4], cmp(Q0, j) + cmp(Q8, j), lap);
        if (LOCAL || SRC) {
            float sv = 0.f;
            if (LOCAL) {
                sv = fmaf(a.a0, cmp(lf0, j), sv);
                if (LOC == 2) {
                    sv = fmaf(a.a1, cmp(lf1, j), sv);
                    sv = fmaf(a.a2, cmp(lf2, j), sv);
                    sv = fmaf(cmp(lcf, j), cmp(lfc, j), sv);
                }
            }
            if (SRC) sv += sj == j ? amp : 0.f;
            lap += sv;
        }
        const float g = gzz * cmp(gxv, j);
        const float pj = cmp(pv, j);
        const float tc = c0v + c0v;
        ov[j] = g * fmaf(cmp(cv, j), lap, fmaf(-g, pj, tc));
        dv[j] = (ov[j] - tc + pj) * a.inv_dt2;
    }
    o = make_float4(ov[0], ov[1], ov[2], ov[3]);
    if (D2) d2 = make_float4(dv[0], dv[1], dv[2], dv[3]);
}
// the packed form where it measured faster: the variants with dense local sources always; the
// plain ones (point source, D2t) only under FWIME_PROP_F32X2_PLAIN
template <int LOC, bool D2, bool SRC>
__device__ __forceinline__ void row_math(const PropArgs &a, const PropK &K, const float4 &L, const float4 &Q0, const float4 &Q1,
                                         const float4 &Q2, const float4 &Q3, const float4 &Q4, const float4 &Q5,
                                         const float4 &Q6, const float4 &Q7, const float4 &Q8, const float4 &Rr,
                                         const float4 &pv, const float4 &cv, const float4 &lf0, const float4 &lf1,
                                         const float4 &lf2, const float4 &lcf, const float4 &lfc, float gzz,
                                         const float4 &gxv, int sj, float amp, float4 &o, float4 &d2)
{
    constexpr bool LOCAL = LOC > 0;
    if constexpr (FWIME_PROP_F32X2 && (LOCAL || FWIME_PROP_F32X2_PLAIN))
        row_math_pk<LOC, D2, SRC>(a, K, L, Q0, Q1, Q2, Q3, Q4, Q5, Q6, Q7, Q8, Rr, pv, cv, lf0, lf1, lf2, lcf, lfc, gzz,
                                    gxv, sj, amp, o, d2);
    else
        row_math_sc<LOC, D2, SRC>(a, L, Q0, Q1, Q2, Q3, Q4, Q5, Q6, Q7, Q8, Rr, pv, cv, lf0, lf1, lf2, lcf, lfc, gzz,
                                    gxv, sj, amp, o, d2);
}

// Adds the injections of the receivers chained from r at one output point: o + c v per receiver, each
// product and sum rounded separately (the arithmetic of a separate injection launch after the step).
__device__ __forceinline__ void inject_point(const PropArgs &a, int shot, int r, float c, float &o)
{
    for (; r >= 0; r = __ldg(a.inj_next + r))
        o = __fadd_rn(o, __fmul_rn(c, __ldg(a.inj_val + (long long)shot * a.inj_vstride + r)));
}

// The time step of one warp's work item (strip, chunk) of shot `shot`; wsm is the warp's shared
// memory (CUR_SLOTS x CUR_ROW + AUX_SLOTS x naux_max x STRIP floats).
template <int LOC, bool D2, bool SRC, bool INJ = false>
__device__ __forceinline__ void prop_body(const PropArgs &a, const int wid, const int shot, float *wsm)
{
    constexpr bool LOCAL = LOC > 0;
    const int lane = threadIdx.x & 31;
    const int strip = wid % a.nstrip, chunk = wid / a.nstrip;
    const int x0 = strip * STRIP;
    const int x = x0 + lane * 4;
    const int z0 = 4 + chunk * a.zchunk;
    const int z1 = min(z0 + a.zchunk, a.NZ - 4);
    const bool xin = x < a.NXP;
    const long long so = (long long)shot * a.P;
    const float *__restrict__ cur = a.cur + so;
    const float *prev = a.prev + so;
    float *out = a.out + so;
    const long long NXP = a.NXP;

    // aux row layout: [prev][c][f0?][f1?][f2?][coef, fc?]
    const int i_f0 = 2, i_f1 = i_f0 + (a.f0 != nullptr), i_f2 = i_f1 + (a.f1 != nullptr),
              i_cf = i_f2 + (a.f2 != nullptr);
    // LOC 1: exactly one local source, f0 (weight a0)
    const int naux = LOC == 2 ? i_cf + (a.fc != nullptr ? 2 : 0) : (LOC == 1 ? 3 : 2);
    float *curR = wsm;
    float *auxR = wsm + CUR_SLOTS * CUR_ROW;

    // copy bounds do not change along the march: hoisted out of the loop
    const int c0 = x0 - 4 + 4 * lane, c1 = x0 - 4 + 4 * (lane + 32);
    const bool ok0 = c0 >= 0 && c0 + 4 <= a.NXP;
    const bool ok1 = lane < CUR_ROW / 4 - 32 && c1 + 4 <= a.NXP;
    auto issue_cur = [&](int zr) {
        if (zr > z1 + 3) return;
        float *dst = curR + ((unsigned)zr % CUR_SLOTS) * CUR_ROW;
        const float *src = cur + (long long)zr * NXP;
        cp16(dst + 4 * lane, ok0 ? src + c0 : cur, ok0);
#if FWIME_PROP_PRED
        cp16p(dst + 4 * (lane + 32), ok1 ? src + c1 : cur, ok1, lane < CUR_ROW / 4 - 32);
#else
        if (lane < CUR_ROW / 4 - 32) cp16(dst + 4 * (lane + 32), ok1 ? src + c1 : cur, ok1);
#endif
    };
    const long long o_x = xin ? x : 0;
    auto issue_aux = [&](int zr) {
        if (zr >= z1) return;
        float *dst = auxR + ((unsigned)zr % AUX_SLOTS) * naux * STRIP + 4 * lane;
        const long long o2 = xin ? (long long)zr * NXP + o_x : 0;
        cp16(dst, prev + o2, xin);
        cp16(dst + STRIP, a.c + o2, xin);
        if (LOCAL) {
            // local sources vanish outside the source rows: zero-filled there, not read
            const bool lin = xin && zr >= a.zs_lo && zr < a.zs_hi;
            if (LOC == 1) {
                cp16(dst + i_f0 * STRIP, a.f0 + so + o2, lin);
            } else {
                if (a.f0) cp16(dst + i_f0 * STRIP, a.f0 + so + o2, lin);
                if (a.f1) cp16(dst + i_f1 * STRIP, a.f1 + so + o2, lin);
                if (a.f2) cp16(dst + i_f2 * STRIP, a.f2 + so + o2, lin);
                if (a.fc) {
                    cp16(dst + i_cf * STRIP, a.coef + o2, lin);
                    cp16(dst + (i_cf + 1) * STRIP, a.fc + so + o2, lin);
                }
            }
        }
    };

    // register queue rows z0-4 .. z0+3
    float4 q[9];
#pragma unroll
    for (int k = 0; k < 8; ++k) q[k] = xin ? ldg4(cur + (long long)(z0 - 4 + k) * NXP + x) : f4zero();
    // prologue: one group per iteration of look-ahead (rows z0 .. z0+3 feed the first x-taps)
#pragma unroll
    for (int g = 0; g < AUX_SLOTS; ++g) {
        if (g < 4) issue_cur(z0 + g);
        issue_cur(z0 + 4 + g);
        issue_aux(z0 + g);
        cp_commit();
    }
    for (int g = AUX_SLOTS; g < 4; ++g) issue_cur(z0 + g);   // (only when the depth is below 4)
    const float4 gxv = xin ? ldg4(a.gx + x) : f4zero();

    long long soff = -1;
    float amp = 0.f;
    if (SRC) {
        soff = a.src_off[shot];
        amp = a.src_amp[(long long)shot * a.src_stride] * a.src_scale;
    }

    // One output row zz; the queue's logical row k (zz-4+k) lives in q[(k + R) % 9], so nine
    // consecutive rows rotate the queue through the registers without moving any of them.
#define FWIME_PROP_ROW(R)                                                                                    \
    {                                                                                                        \
        const int zz = z + (R);                                                                              \
        cp_wait<AUX_SLOTS - 1>();                                                                            \
        __syncwarp();                                                                                        \
        const float *crow = curR + ((unsigned)zz % CUR_SLOTS) * CUR_ROW;                                     \
        q[(8 + (R)) % 9] = lds4(curR + ((unsigned)(zz + 4) % CUR_SLOTS) * CUR_ROW + 4 + 4 * lane);           \
        const float4 L = lds4(crow + 4 * lane);                                                              \
        const float4 Rr = lds4(crow + 8 + 4 * lane);                                                         \
        const float *arow = auxR + ((unsigned)zz % AUX_SLOTS) * naux * STRIP + 4 * lane;                     \
        const float4 pv = lds4(arow);                                                                        \
        const float4 cv = lds4(arow + STRIP);                                                                \
        float4 lf0 = f4zero(), lf1 = f4zero(), lf2 = f4zero(), lcf = f4zero(), lfc = f4zero();               \
        if (LOC == 1) {                                                                                      \
            lf0 = lds4(arow + i_f0 * STRIP);                                                                 \
        } else if (LOC == 2) {                                                                               \
            if (a.f0) lf0 = lds4(arow + i_f0 * STRIP);                                                       \
            if (a.f1) lf1 = lds4(arow + i_f1 * STRIP);                                                       \
            if (a.f2) lf2 = lds4(arow + i_f2 * STRIP);                                                       \
            if (a.fc) { lcf = lds4(arow + i_cf * STRIP); lfc = lds4(arow + (i_cf + 1) * STRIP); }            \
        }                                                                                                    \
        const long long idx = (long long)zz * NXP + x;                                                       \
        const float gzz = __ldg(a.gz + zz);                                                                  \
        int sj = -1; /* the point source's column within this lane's four, if it is in them */              \
        if (SRC) {                                                                                           \
            const long long sd = soff - idx;                                                                 \
            sj = (sd >= 0 && sd < 4) ? (int)sd : -1;                                                         \
        }                                                                                                    \
        float4 o, d2;                                                                                        \
        row_math<LOC, D2, SRC>(a, prop_k(a), L, q[(0 + (R)) % 9], q[(1 + (R)) % 9], q[(2 + (R)) % 9], q[(3 + (R)) % 9], \
                                 q[(4 + (R)) % 9], q[(5 + (R)) % 9], q[(6 + (R)) % 9], q[(7 + (R)) % 9],      \
                                 q[(8 + (R)) % 9], Rr, pv, cv, lf0, lf1, lf2, lcf, lfc, gzz, gxv, sj, amp, o, d2); \
        if (xin) {                                                                                           \
            st4(out + idx, o);                                                                               \
            if (D2 && zz >= a.zs_lo && zz < a.zs_hi) st4(a.d2 + so + idx, d2);                               \
        }                                                                                                    \
        __syncwarp(); /* every lane is done with this row's slots before they are refilled */              \
        issue_cur(zz + 4 + AUX_SLOTS);                                                                       \
        issue_aux(zz + AUX_SLOTS);                                                                           \
        cp_commit();                                                                                         \
    }

    int z = z0;
    for (; z + 9 <= z1; z += 9) {
        FWIME_PROP_ROW(0) FWIME_PROP_ROW(1) FWIME_PROP_ROW(2) FWIME_PROP_ROW(3) FWIME_PROP_ROW(4)
        FWIME_PROP_ROW(5) FWIME_PROP_ROW(6) FWIME_PROP_ROW(7) FWIME_PROP_ROW(8)
    }
    for (; z < z1; ++z) {   // the last (z1 - z0) mod 9 rows: shift the queue by one register per row
        FWIME_PROP_ROW(0)
#pragma unroll
        for (int k = 0; k < 8; ++k) q[k] = q[k + 1];
    }
#undef FWIME_PROP_ROW
    cp_wait<0>();
    if (INJ && xin) {
        // receivers in this warp's rows: each lane adds the injection to the outputs it wrote itself (read
        // back by the writing thread), after the march so the loop above keeps its registers
        const int zlo = max(z0, a.inj_lo), zhi = min(z1, a.inj_hi);
        for (int zz = zlo; zz < zhi; ++zz) {
            const int4 m4 = *reinterpret_cast<const int4 *>(a.inj_map + (long long)(zz - a.inj_lo) * NXP + x);
            if ((m4.x & m4.y & m4.z & m4.w) < 0) continue;   // none of the lane's four points
            const long long idx = (long long)zz * NXP + x;
            const float4 o0 = *reinterpret_cast<const float4 *>(out + idx);
            float4 o = o0;
            const float4 cv = ldg4(a.c + idx);
            inject_point(a, shot, m4.x, cv.x, o.x);
            inject_point(a, shot, m4.y, cv.y, o.y);
            inject_point(a, shot, m4.z, cv.z, o.z);
            inject_point(a, shot, m4.w, cv.w, o.w);
            st4(out + idx, o);
            if (D2 && zz >= a.zs_lo && zz < a.zs_hi) {
                // the D2t output gains the injection too: d2 + (o - o0) / dt^2
                float *dp = a.d2 + so + idx;
                float4 d = *reinterpret_cast<const float4 *>(dp);
                d.x = fmaf(o.x - o0.x, a.inv_dt2, d.x);
                d.y = fmaf(o.y - o0.y, a.inv_dt2, d.y);
                d.z = fmaf(o.z - o0.z, a.inv_dt2, d.z);
                d.w = fmaf(o.w - o0.w, a.inv_dt2, d.w);
                st4(dp, d);
            }
        }
    }
}

// INJ: the receivers' injection into the output (the adjoint step; LOC = 0, no point source; with D2 the
// injection reaches the D2t output as well)
template <int LOC, bool D2, bool SRC, bool INJ = false>
__global__ void __launch_bounds__(PROP_WARPS * 32, LOC == 2 ? FWIME_PROP_MIN_BLOCKS : (LOC == 1 ? FWIME_PROP_MINB_LOC1 : FWIME_PROP_MINB_PLAIN)) k_prop(const PropArgs a)
{
    extern __shared__ float4 smem4[];
    if (a.rec_d && blockIdx.x == 0) {         // receivers of the input field (the previous step's output)
        const long long s = blockIdx.y;
        for (int r = threadIdx.x; r < a.nrec; r += PROP_WARPS * 32) {
            const float val = a.cur[s * a.P + a.rec_off[r]];
            float *dp = a.rec_d + s * a.rec_dstride + r;
            *dp = a.rec_acc ? *dp + val : val;
        }
    }
    const int wic = threadIdx.x >> 5;
    const int wid = blockIdx.x * PROP_WARPS + wic;
    if (wid >= a.nstrip * a.nchunk) return;   // warp-uniform
    float *wsm = reinterpret_cast<float *>(smem4) + wic * (CUR_SLOTS * CUR_ROW + AUX_SLOTS * a.naux_max * STRIP);
    prop_body<LOC, D2, SRC, INJ>(a, wid, blockIdx.y, wsm);
}

// ------------------------------------------------------------- grouped forward
// One launch advances one time step of every member of a group of shot batches on grids of
// different sizes (and different record lengths): CTA b belongs to the member whose cta_begin is
// the largest <= b.  Members are sorted by decreasing nt, so the members still running at a step
// are a prefix and the grid covers exactly their CTAs.
__global__ void __launch_bounds__(PROP_WARPS * 32, 4) k_prop_group(const GroupMember *__restrict__ m, int nactive, int step)
{
    extern __shared__ float4 smem4[];
    __shared__ PropArgs sa;
    int lo = 0, hi = nactive - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (m[mid].cta_begin <= (int)blockIdx.x) lo = mid; else hi = mid - 1;
    }
    if (threadIdx.x == 0) {
        sa = m[lo].a[step & 1];
        sa.src_amp += step;
    }
    __syncthreads();
    const int local = (int)blockIdx.x - m[lo].cta_begin;
    const int cps = m[lo].ctas_per_shot;
    const int shot = local / cps;
    const int wic = threadIdx.x >> 5;
    const int wid = (local - shot * cps) * PROP_WARPS + wic;
    if (wid >= sa.nstrip * sa.nchunk) return;   // warp-uniform
    float *wsm = reinterpret_cast<float *>(smem4) + wic * (CUR_SLOTS * CUR_ROW + AUX_SLOTS * 2 * STRIP);
    prop_body<0, false, true>(sa, wid, shot, wsm);
}

// after step n the new field q^{n+1} of a member is in buffer B for even n, A for odd n
__global__ void k_points_group(const GroupRec *__restrict__ g, int nactive, int step)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    int lo = 0, hi = nactive - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (g[mid].rec_begin <= i) lo = mid; else hi = mid - 1;
    }
    const GroupRec &r = g[lo];
    const int local = i - r.rec_begin;
    if (local >= r.nshot * r.nrec) return;
    const int s = local / r.nrec, k = local - s * r.nrec;
    const float *f = (step & 1) ? r.fA : r.fB;
    r.d[(long long)s * r.nt * r.nrec + (long long)(step + 1) * r.nrec + k] = f[(long long)s * r.P + r.rec_off[k]];
}

cudaError_t launch_prop_group(const GroupMember *m, int nactive, int ctas, const GroupRec *g, int nrec_threads,
                              int step, cudaStream_t st, bool record)
{
    const size_t smem = (size_t)PROP_WARPS * (CUR_SLOTS * CUR_ROW + AUX_SLOTS * 2 * STRIP) * sizeof(float);
    if (!record) {
        k_prop_group<<<ctas, PROP_WARPS * 32, smem, st>>>(m, nactive, step);
    } else {
        k_points_group<<<(nrec_threads + 127) / 128, 128, 0, st>>>(g, nactive, step);
    }
    return cudaGetLastError();
}

template <int LOC, bool D2, bool SRC, bool INJ = false>
static void launch_prop_t(const PropArgs &a, dim3 grid, dim3 block, size_t smem, cudaStream_t st)
{
    // once per instantiation, thread-safe (function-local static)
    static const cudaError_t attr =
        cudaFuncSetAttribute(k_prop<LOC, D2, SRC, INJ>, cudaFuncAttributeMaxDynamicSharedMemorySize, 100 * 1024);
    (void)attr;
    k_prop<LOC, D2, SRC, INJ><<<grid, block, smem, st>>>(a);
}

// Resident CTAs per SM of the plain (no local source) variant with the smem it launches with.
cudaError_t prop_occupancy(int *blocks_per_sm)
{
    const size_t smem = (size_t)PROP_WARPS * (CUR_SLOTS * CUR_ROW + AUX_SLOTS * 2 * STRIP) * sizeof(float);
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, k_prop<0, false, false>, PROP_WARPS * 32,
                                                         smem);
}

cudaError_t launch_prop(const PropArgs &a0, int nshot, cudaStream_t st)
{
    PropArgs a = a0;
    prop_pairs(a);
    const int nwarps = a.nstrip * a.nchunk;
    dim3 grid((nwarps + PROP_WARPS - 1) / PROP_WARPS, nshot);
    dim3 block(PROP_WARPS * 32);
    const bool local = a.f0 || a.f1 || a.f2 || a.fc;
    const bool d2 = a.d2 != nullptr;
    const bool src = a.src_off != nullptr;
    a.naux_max = 2 + (local ? (a.f0 != nullptr) + (a.f1 != nullptr) + (a.f2 != nullptr) + (a.fc ? 2 : 0) : 0);
    const size_t smem = (size_t)PROP_WARPS * (CUR_SLOTS * CUR_ROW + AUX_SLOTS * a.naux_max * STRIP) * sizeof(float);
    const int loc = !local ? 0 : (a.f1 || a.f2 || a.fc || !a.f0) ? 2 : 1;
    const int key = loc * 4 + (d2 ? 2 : 0) + (src ? 1 : 0);
    if (a.inj_val) {                           // the caller injects only into plain steps, with or without D2t
        if (key != 0 && key != 2) return cudaErrorInvalidValue;
        if (d2) launch_prop_t<0, true, false, true>(a, grid, block, smem, st);
        else launch_prop_t<0, false, false, true>(a, grid, block, smem, st);
        return cudaGetLastError();
    }
    switch (key) {
    case 0: launch_prop_t<0, false, false>(a, grid, block, smem, st); break;
    case 1: launch_prop_t<0, false, true>(a, grid, block, smem, st); break;
    case 2: launch_prop_t<0, true, false>(a, grid, block, smem, st); break;
    case 3: launch_prop_t<0, true, true>(a, grid, block, smem, st); break;
    case 4: launch_prop_t<1, false, false>(a, grid, block, smem, st); break;
    case 5: launch_prop_t<1, false, true>(a, grid, block, smem, st); break;
    case 6: launch_prop_t<1, true, false>(a, grid, block, smem, st); break;
    case 7: launch_prop_t<1, true, true>(a, grid, block, smem, st); break;
    case 8: launch_prop_t<2, false, false>(a, grid, block, smem, st); break;
    case 9: launch_prop_t<2, false, true>(a, grid, block, smem, st); break;
    case 10: launch_prop_t<2, true, false>(a, grid, block, smem, st); break;
    default: launch_prop_t<2, true, true>(a, grid, block, smem, st); break;
    }
    return cudaGetLastError();
}

// ----------------------------------------------------------------- points
// Receiver recording d[n][r] = q^n(rec_r) and adjoint injection of the data
// residual at the receivers (the transpose of recording, scaled by c g so it
// enters the mu-form adjoint recursion inside c (L mu + R^T r)).
__global__ void k_points(const PointsArgs a)
{
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    const int s = blockIdx.y;
    if (r >= a.nrec) return;
    const long long off = (long long)s * a.P + a.rec_off[r];
    if (a.d) {
        float val = a.f1[off];
        if (a.f2) val += a.f2[off];
        float *dp = a.d + (long long)s * a.dstride + r;
        *dp = a.accumulate ? *dp + val : val;
    }
    if (a.fld) atomicAdd(a.fld + off, a.c[a.rec_off[r]] * a.val[(long long)s * a.vstride + r]);
}

cudaError_t launch_points(const PointsArgs &a, int nshot, cudaStream_t st)
{
    dim3 grid((a.nrec + 127) / 128, nshot);
    k_points<<<grid, 128, 0, st>>>(a);
    return cudaGetLastError();
}

}  // namespace fwk
