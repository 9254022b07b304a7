// Two time steps of the wave equation per launch (temporal blocking of the stencil of k_prop.cu):
//
//   q^{n+1} = g (2 q^n     - g q^{n-1} + c (L q^n     + s^n))
//   q^{n+2} = g (2 q^{n+1} - g q^n     + c (L q^{n+1} + s^{n+1}))
//
// with the same arithmetic, point by point and in the same order, as two launches of k_prop (whose
// packed two-lane form rounds every operation as this scalar form does), so the results are identical.  Each launch reads q^n and q^{n-1} and writes q^{n+1} and q^{n+2}: 16 bytes
// per two updates of a shot-point instead of 24 (plus one D2t field per step and one local-source field
// per step when the variant has them).
//
// A warp marches down z over a strip of 128 columns (32 lanes x float4) with two 9-row register queues:
// q^n (rows zz-4 .. zz+4, fed from a cp.async ring as in k_prop) for the first step at row zz, and
// q^{n+1} (rows zz-8 .. zz) for the second step at row zz-4, whose x-neighbours come from the adjacent
// lanes by shuffles.  Strips therefore overlap: a warp owns (writes) only the 120 inner columns, lanes 0
// and 31 computing q^{n+1} for the neighbours' edge columns; a chunk of output rows [z0, z1) computes
// q^{n+1} on rows z0-4 .. z1+3.  Outputs go to two buffers distinct from the inputs (neighbouring warps
// still read q^n and q^{n-1} at these columns).
#include "fwime_kernels.cuh"

namespace fwk {

namespace {
__device__ __forceinline__ float4 z4() { return make_float4(0.f, 0.f, 0.f, 0.f); }
__device__ __forceinline__ float4 g4(const float *p) { return __ldg(reinterpret_cast<const float4 *>(p)); }
__device__ __forceinline__ void s4(float *p, float4 v) { *reinterpret_cast<float4 *>(p) = v; }
__device__ __forceinline__ float4 l4(const float *p) { return *reinterpret_cast<const float4 *>(p); }
__device__ __forceinline__ float c4(const float4 &v, int j) { return j == 0 ? v.x : (j == 1 ? v.y : (j == 2 ? v.z : v.w)); }
__device__ __forceinline__ float4 up4(float4 v)
{
    v.x = __shfl_up_sync(0xffffffffu, v.x, 1); v.y = __shfl_up_sync(0xffffffffu, v.y, 1);
    v.z = __shfl_up_sync(0xffffffffu, v.z, 1); v.w = __shfl_up_sync(0xffffffffu, v.w, 1);
    return v;
}
__device__ __forceinline__ float4 dn4(float4 v)
{
    v.x = __shfl_down_sync(0xffffffffu, v.x, 1); v.y = __shfl_down_sync(0xffffffffu, v.y, 1);
    v.z = __shfl_down_sync(0xffffffffu, v.z, 1); v.w = __shfl_down_sync(0xffffffffu, v.w, 1);
    return v;
}
__device__ __forceinline__ void cpa(float *dst, const float *src, bool valid)
{
    const unsigned d = static_cast<unsigned>(__cvta_generic_to_shared(dst));
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(d), "l"(src), "r"(valid ? 16 : 0) : "memory");
}
__device__ __forceinline__ void cpc() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cpw() { asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory"); }
}  // namespace

constexpr int P2_STRIP = 120;                  // owned columns per warp
constexpr int P2_CUR_SLOTS = 8, P2_AUX_SLOTS = 4;
constexpr int P2_ROW = STRIP + 8;              // q^n row with +-4 halo

// one grid point of one step: o = g (2 c0 - g p + cv (lap + sv)), lap from the 12 x-samples rr (the lane's
// 4 points and 4 on each side) and the z-samples of the 9-row queue
#define FWIME_P2_LAP(rr, Q0, Q1, Q2, Q3, Q5, Q6, Q7, Q8, j, lap)                                         \
    {                                                                                                   \
        lap = axc * rr[(j) + 4];                                                                        \
        lap = fmaf(a.ax[1], rr[(j) + 3] + rr[(j) + 5], lap);                                            \
        lap = fmaf(a.ax[2], rr[(j) + 2] + rr[(j) + 6], lap);                                            \
        lap = fmaf(a.ax[3], rr[(j) + 1] + rr[(j) + 7], lap);                                            \
        lap = fmaf(a.ax[4], rr[(j) + 0] + rr[(j) + 8], lap);                                            \
        lap = fmaf(a.az[1], c4(Q3, j) + c4(Q5, j), lap);                                                \
        lap = fmaf(a.az[2], c4(Q2, j) + c4(Q6, j), lap);                                                \
        lap = fmaf(a.az[3], c4(Q1, j) + c4(Q7, j), lap);                                                \
        lap = fmaf(a.az[4], c4(Q0, j) + c4(Q8, j), lap);                                                \
    }

template <bool LOCAL, bool D2, bool SRC>
__device__ __forceinline__ void prop2_body(const Prop2Args &a, const int wid, const int shot, float *wsm)
{
    const int lane = threadIdx.x & 31;
    const int strip = wid % a.nstrip, chunk = wid / a.nstrip;
    const int x0 = strip * P2_STRIP - 4;        // first column of the 128-column stage-1 strip (multiple of 4)
    const int x = x0 + lane * 4;
    const bool xin = x >= 0 && x < a.NXP;       // stage-1 columns inside the row
    const bool own = lane >= 1 && lane <= 30 && xin;   // owned (written) columns
    const int z0 = 4 + chunk * a.zchunk;
    const int z1 = min(z0 + a.zchunk, a.NZ - 4);
    const long long so = (long long)shot * a.P;
    const float *__restrict__ cur = a.cur + so;
    const float *prev = a.prev + so;
    const long long NXP = a.NXP;
    // aux row layout for iteration zz: [prev(zz)][c(zz)][f(zz), n][c(zz-4)][f(zz-4), n+1]
    const int naux = LOCAL ? 5 : 3;
    float *curR = wsm;
    float *auxR = wsm + P2_CUR_SLOTS * P2_ROW;

    const int cc0 = x0 - 4 + 4 * lane, cc1 = x0 - 4 + 4 * (lane + 32);
    const bool ok0 = cc0 >= 0 && cc0 + 4 <= a.NXP;
    const bool ok1 = lane < P2_ROW / 4 - 32 && cc1 >= 0 && cc1 + 4 <= a.NXP;
    // q^n rows needed: z0-8 .. z1+7 (rows outside [0, NZ) read as zero)
    auto issue_cur = [&](int zr) {
        if (zr > z1 + 7) return;
        const bool rin = zr >= 0 && zr < a.NZ;
        float *dst = curR + ((unsigned)(zr + 16) % P2_CUR_SLOTS) * P2_ROW;
        const float *src = cur + (long long)(rin ? zr : 0) * NXP;
        cpa(dst + 4 * lane, (ok0 && rin) ? src + cc0 : cur, ok0 && rin);
        if (lane < P2_ROW / 4 - 32) cpa(dst + 4 * (lane + 32), (ok1 && rin) ? src + cc1 : cur, ok1 && rin);
    };
    const long long o_x = xin ? x : 0;
    auto issue_aux = [&](int zz) {   // iteration zz: stage 1 at row zz, stage 2 at row zz - 4
        if (zz > z1 + 3) return;
        float *dst = auxR + ((unsigned)(zz + 16) % P2_AUX_SLOTS) * naux * STRIP + 4 * lane;
        const bool r1 = zz >= 0 && zz < a.NZ, r2 = zz - 4 >= z0 && zz - 4 < z1;
        const long long o1 = (long long)(r1 ? zz : 0) * NXP + o_x, o2 = (long long)(r2 ? zz - 4 : 0) * NXP + o_x;
        cpa(dst, prev + o1, xin && r1);
        cpa(dst + STRIP, a.c + o1, xin && r1);
        cpa(dst + 2 * STRIP, a.c + o2, xin && r2);
        if (LOCAL) {
            cpa(dst + 3 * STRIP, a.f0 + so + o1, xin && r1);
            cpa(dst + 4 * STRIP, a.f1 + so + o2, xin && r2);
        }
    };

    const int zs = z0 - 4;                     // first stage-1 row
    float4 q[9], p[9];                         // q^n rows zz-4..zz+4; q^{n+1} rows zz-8..zz
#pragma unroll
    for (int k = 0; k < 8; ++k) {
        const int zr = zs - 4 + k;
        q[k] = (xin && zr >= 0 && zr < a.NZ) ? g4(cur + (long long)zr * NXP + x) : z4();
    }
#pragma unroll
    for (int k = 0; k < 9; ++k) p[k] = z4();
#pragma unroll
    for (int g = 0; g < P2_AUX_SLOTS; ++g) {
        issue_cur(zs + g);
        issue_cur(zs + 4 + g);
        issue_aux(zs + g);
        cpc();
    }
    const float4 gxv = xin ? g4(a.gx + x) : z4();
    long long soff = -1;
    float amp0 = 0.f, amp1 = 0.f;
    if (SRC) {
        soff = a.src_off[shot];
        amp0 = a.src_amp[(long long)shot * a.src_stride] * a.src_scale;
        amp1 = a.src_amp[(long long)shot * a.src_stride + 1] * a.src_scale;
    }
    const float axc = a.ax[0] + a.az[0];

    // iteration zz: stage 1 (row zz) then stage 2 (row zz-4); logical queue row k of q is q[(k+R)%9],
    // of p is p[(k+R)%9] (p's logical row 8 = the row just computed)
#define FWIME_P2_ROW(R)                                                                                      \
    {                                                                                                        \
        const int zz = z + (R);                                                                              \
        cpw<P2_AUX_SLOTS - 1>();                                                                             \
        __syncwarp();                                                                                        \
        const float *crow = curR + ((unsigned)(zz + 16) % P2_CUR_SLOTS) * P2_ROW;                            \
        q[(8 + (R)) % 9] = l4(curR + ((unsigned)(zz + 20) % P2_CUR_SLOTS) * P2_ROW + 4 + 4 * lane);          \
        const float4 L1 = l4(crow + 4 * lane), R1 = l4(crow + 8 + 4 * lane);                                 \
        const float *arow = auxR + ((unsigned)(zz + 16) % P2_AUX_SLOTS) * naux * STRIP + 4 * lane;           \
        const float4 pv = l4(arow), cv1 = l4(arow + STRIP), cv2 = l4(arow + 2 * STRIP);                      \
        float4 f1v = z4(), f2v = z4();                                                                       \
        if (LOCAL) { f1v = l4(arow + 3 * STRIP); f2v = l4(arow + 4 * STRIP); }                               \
        const float4 Q0 = q[(0 + (R)) % 9], Q1 = q[(1 + (R)) % 9], Q2 = q[(2 + (R)) % 9],                    \
                     Q3 = q[(3 + (R)) % 9], Q4 = q[(4 + (R)) % 9], Q5 = q[(5 + (R)) % 9],                    \
                     Q6 = q[(6 + (R)) % 9], Q7 = q[(7 + (R)) % 9], Q8 = q[(8 + (R)) % 9];                    \
        const bool r1 = zz >= 0 && zz < a.NZ;                                                                \
        const float gz1 = r1 ? __ldg(a.gz + zz) : 0.f;                                                       \
        const long long i1 = (long long)(r1 ? zz : 0) * NXP + x;                                             \
        float n1[4], d1[4];                                                                                  \
        {                                                                                                    \
            const float rr[12] = {L1.x, L1.y, L1.z, L1.w, Q4.x, Q4.y, Q4.z, Q4.w, R1.x, R1.y, R1.z, R1.w};   \
            _Pragma("unroll") for (int j = 0; j < 4; ++j) {                                                  \
                const float c0v = rr[j + 4];                                                                 \
                float lap;                                                                                   \
                FWIME_P2_LAP(rr, Q0, Q1, Q2, Q3, Q5, Q6, Q7, Q8, j, lap)                                     \
                if (LOCAL || SRC) {                                                                           \
                    float sv = 0.f;                                                                          \
                    if (LOCAL) sv = fmaf(a.a0, c4(f1v, j), sv);                                              \
                    if (SRC) sv += (xin && soff == i1 + j) ? amp0 : 0.f;                                     \
                    lap += sv;                                                                               \
                }                                                                                            \
                const float g = gz1 * c4(gxv, j);                                                            \
                const float pj = c4(pv, j);                                                                  \
                const float tc = c0v + c0v;                                                                  \
                n1[j] = g * fmaf(c4(cv1, j), lap, fmaf(-g, pj, tc));                                         \
                d1[j] = (n1[j] - tc + pj) * a.inv_dt2;                                                       \
            }                                                                                                \
        }                                                                                                    \
        p[(8 + (R)) % 9] = make_float4(n1[0], n1[1], n1[2], n1[3]);                                          \
        if (own && zz >= z0 && zz < z1) {                                                                    \
            s4(a.out1 + so + i1, p[(8 + (R)) % 9]);                                                          \
            if (D2) s4(a.d2a + so + i1, make_float4(d1[0], d1[1], d1[2], d1[3]));                            \
        }                                                                                                    \
        const float4 P4 = p[(4 + (R)) % 9];                                                                  \
        const float4 PL = up4(P4), PR = dn4(P4);                                                             \
        const int z2 = zz - 4;                                                                               \
        if (z2 >= z0 && z2 < z1) {                                                                           \
            const float4 P0 = p[(0 + (R)) % 9], P1 = p[(1 + (R)) % 9], P2 = p[(2 + (R)) % 9],                \
                         P3 = p[(3 + (R)) % 9], P5 = p[(5 + (R)) % 9], P6 = p[(6 + (R)) % 9],                \
                         P7 = p[(7 + (R)) % 9], P8 = p[(8 + (R)) % 9];                                       \
            const float rr[12] = {PL.x, PL.y, PL.z, PL.w, P4.x, P4.y, P4.z, P4.w, PR.x, PR.y, PR.z, PR.w};   \
            const float gz2 = __ldg(a.gz + z2);                                                              \
            const long long i2 = (long long)z2 * NXP + x;                                                    \
            float n2[4], d2v[4];                                                                             \
            _Pragma("unroll") for (int j = 0; j < 4; ++j) {                                                  \
                const float c0v = rr[j + 4];                                                                 \
                float lap;                                                                                   \
                FWIME_P2_LAP(rr, P0, P1, P2, P3, P5, P6, P7, P8, j, lap)                                     \
                if (LOCAL || SRC) {                                                                                  \
                    float sv = 0.f;                                                                                  \
                    if (LOCAL) sv = fmaf(a.a0, c4(f2v, j), sv);                                                      \
                    if (SRC) sv += (xin && soff == i2 + j) ? amp1 : 0.f;                                             \
                    lap += sv;                                                                                       \
                }                                                                                                    \
                const float g = gz2 * c4(gxv, j);                                                                    \
                const float pj = c4(Q0, j);                                                                          \
                const float tc = c0v + c0v;                                                                          \
                n2[j] = g * fmaf(c4(cv2, j), lap, fmaf(-g, pj, tc));                                                 \
                d2v[j] = (n2[j] - tc + pj) * a.inv_dt2;                                                              \
            }                                                                                                \
            if (own) {                                                                                       \
                s4(a.out2 + so + i2, make_float4(n2[0], n2[1], n2[2], n2[3]));                               \
                if (D2) s4(a.d2b + so + i2, make_float4(d2v[0], d2v[1], d2v[2], d2v[3]));                    \
            }                                                                                                \
        }                                                                                                    \
        __syncwarp();                                                                                        \
        issue_cur(zz + 4 + P2_AUX_SLOTS);                                                                    \
        issue_aux(zz + P2_AUX_SLOTS);                                                                        \
        cpc();                                                                                               \
    }

    int z = zs;
    const int zend = z1 + 4;                   // last stage-1 row is z1 + 3
    for (; z + 9 <= zend; z += 9) {
        FWIME_P2_ROW(0) FWIME_P2_ROW(1) FWIME_P2_ROW(2) FWIME_P2_ROW(3) FWIME_P2_ROW(4)
        FWIME_P2_ROW(5) FWIME_P2_ROW(6) FWIME_P2_ROW(7) FWIME_P2_ROW(8)
    }
    for (; z < zend; ++z) {
        FWIME_P2_ROW(0)
#pragma unroll
        for (int k = 0; k < 8; ++k) { q[k] = q[k + 1]; p[k] = p[k + 1]; }
    }
#undef FWIME_P2_ROW
    cpw<0>();
}
#undef FWIME_P2_LAP

template <bool LOCAL, bool D2, bool SRC>
__global__ void __launch_bounds__(PROP_WARPS * 32) k_prop2(const Prop2Args a)
{
    extern __shared__ float4 smem4[];
    const int wic = threadIdx.x >> 5;
    const int wid = blockIdx.x * PROP_WARPS + wic;
    if (wid >= a.nstrip * a.nchunk) return;   // warp-uniform
    constexpr int naux = LOCAL ? 5 : 3;
    float *wsm = reinterpret_cast<float *>(smem4) + wic * (P2_CUR_SLOTS * P2_ROW + P2_AUX_SLOTS * naux * STRIP);
    prop2_body<LOCAL, D2, SRC>(a, wid, blockIdx.y, wsm);
}

template <bool LOCAL, bool D2, bool SRC>
static void launch_prop2_t(const Prop2Args &a, int nshot, cudaStream_t st)
{
    constexpr int naux = LOCAL ? 5 : 3;
    const size_t smem = (size_t)PROP_WARPS * (P2_CUR_SLOTS * P2_ROW + P2_AUX_SLOTS * naux * STRIP) * sizeof(float);
    static bool attr = false;
    if (!attr) {
        cudaFuncSetAttribute(k_prop2<LOCAL, D2, SRC>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        attr = true;
    }
    const int nwarps = a.nstrip * a.nchunk;
    k_prop2<LOCAL, D2, SRC><<<dim3((nwarps + PROP_WARPS - 1) / PROP_WARPS, nshot), PROP_WARPS * 32, smem, st>>>(a);
}

int prop2_strips(int NXP) { return (NXP + P2_STRIP - 1) / P2_STRIP; }

cudaError_t launch_prop2(const Prop2Args &a, int nshot, cudaStream_t st)
{
    const bool local = a.f0 != nullptr, d2 = a.d2a != nullptr, src = a.src_off != nullptr;
    const int key = (local ? 4 : 0) | (d2 ? 2 : 0) | (src ? 1 : 0);
    switch (key) {
    case 0: launch_prop2_t<false, false, false>(a, nshot, st); break;
    case 1: launch_prop2_t<false, false, true>(a, nshot, st); break;
    case 2: launch_prop2_t<false, true, false>(a, nshot, st); break;
    case 3: launch_prop2_t<false, true, true>(a, nshot, st); break;
    case 4: launch_prop2_t<true, false, false>(a, nshot, st); break;
    case 5: launch_prop2_t<true, false, true>(a, nshot, st); break;
    case 6: launch_prop2_t<true, true, false>(a, nshot, st); break;
    default: launch_prop2_t<true, true, true>(a, nshot, st); break;
    }
    return cudaGetLastError();
}

}  // namespace fwk
