// fwime_forward_static: the nonlinear forward modelling f(m) for callers that
// cannot allocate device memory.
//
// Some callers cannot call cudaMalloc at all: code that runs inside another
// framework's memory pool or allocator hooks, a process whose device memory is
// reserved up front, or a host thread that must never block on the driver's
// allocator.  For them this entry point takes no context (creating one
// allocates) and allocates nothing: its scratch -- the padded model c, b, the
// sponge tables, the receiver/source offsets, a status word and two wavefields
// per shot -- lives in one file-scope __device__ array of
// FWIME_STATIC_SCRATCH_BYTES that every GPU loading the library holds until the
// process exits.  The caller still passes the inputs (v, w) and the output (d)
// as device pointers.
//
// The array's host-side name is only a stand-in, not a device address.  Every
// call looks the address up with cudaGetSymbolAddress on the device that is
// current at the time (the lookup allocates nothing), so the address is never
// stale after a device reset or under another context.  Every call shares the
// array and leaves its contents behind; the wavefields and the status word are
// cleared at the start of each call.  Calls whose work overlaps on the GPU (two
// streams, or two host threads) race on the array and must be serialised by
// the caller.
//
// The model check (positive velocity below the stability bound) runs on the
// device; the call copies the offsets in from host memory, waits for the check
// on its stream and returns FWIME_ECFL before any time step when it fails.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdio>
#include <cstring>
#include <vector>

#include "../../include/fwime.h"
#include "fwime_kernels.cuh"

using namespace fwk;

static constexpr size_t SCRATCH_FLOATS = FWIME_STATIC_SCRATCH_BYTES / sizeof(float);
static __device__ __align__(256) float g_scratch[SCRATCH_FLOATS];

namespace {
thread_local char g_err[256] = {0};

size_t al(size_t n) { return (n + 63) & ~(size_t)63; }   // 256-byte granules

// Device address of the scratch array on the current device (looked up on every call).
int scratch_ptr(float **out)
{
    void *p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_scratch);
    if (e != cudaSuccess || !p) {
        cudaGetLastError();
        snprintf(g_err, sizeof(g_err), "cudaGetSymbolAddress(scratch): %s", cudaGetErrorString(e));
        return FWIME_ECUDA;
    }
    *out = static_cast<float *>(p);
    return FWIME_OK;
}
}  // namespace

extern "C" size_t fwime_static_scratch_bytes(const fwime_grid *g, const fwime_geom *geo)
{
    if (!g || !geo || g->nz < 1 || g->nx < 1 || g->sponge < 0 || geo->nshot < 1 || geo->nrec < 1) return 0;
    const int o = g->sponge + 4, NZ = g->nz + 2 * o, NX = g->nx + 2 * o, NXP = (NX + 31) / 32 * 32;
    const size_t P = (size_t)NZ * NXP;
    const size_t floats = al(P) * (2 + 2 * (size_t)geo->nshot) + al(NZ) + al(NXP) + al(geo->nshot + geo->nrec + 1);
    return floats * sizeof(float);
}

extern "C" int fwime_forward_static(const fwime_grid *g, const fwime_geom *geo, const float *v, const float *w,
                                    float *d, void *cuda_stream)
{
    g_err[0] = 0;
    if (!g || !geo || !v || !w || !d) {
        snprintf(g_err, sizeof(g_err), "fwime_forward_static: null argument");
        return FWIME_EINVAL;
    }
    if (g->nz < 1 || g->nx < 1 || g->sponge < 0 || g->nt < 2 || !(g->dx > 0.f) || !(g->dz > 0.f) ||
        !(g->dt > 0.f) || geo->nshot < 1 || geo->nrec < 1 || !geo->src_iz || !geo->src_ix || !geo->rec_iz ||
        !geo->rec_ix) {
        snprintf(g_err, sizeof(g_err), "fwime_forward_static: invalid grid or geometry");
        return FWIME_EINVAL;
    }
    for (int s = 0; s < geo->nshot; ++s)
        if (geo->src_iz[s] < 0 || geo->src_iz[s] >= g->nz || geo->src_ix[s] < 0 || geo->src_ix[s] >= g->nx) {
            snprintf(g_err, sizeof(g_err), "fwime_forward_static: source %d outside the grid", s);
            return FWIME_EINVAL;
        }
    for (int r = 0; r < geo->nrec; ++r)
        if (geo->rec_iz[r] < 0 || geo->rec_iz[r] >= g->nz || geo->rec_ix[r] < 0 || geo->rec_ix[r] >= g->nx) {
            snprintf(g_err, sizeof(g_err), "fwime_forward_static: receiver %d outside the grid", r);
            return FWIME_EINVAL;
        }
    const size_t need = fwime_static_scratch_bytes(g, geo);
    if (need > FWIME_STATIC_SCRATCH_BYTES) {
        snprintf(g_err, sizeof(g_err),
                 "fwime_forward_static: problem needs %zu bytes of scratch, the static array holds %zu",
                 need, (size_t)FWIME_STATIC_SCRATCH_BYTES);
        return FWIME_ENOMEM;
    }
    float *base = nullptr;
    const int rc = scratch_ptr(&base);
    if (rc != FWIME_OK) return rc;
    cudaStream_t st = reinterpret_cast<cudaStream_t>(cuda_stream);

    const int o = g->sponge + 4, NZ = g->nz + 2 * o, NX = g->nx + 2 * o, NXP = (NX + 31) / 32 * 32;
    const long long P = (long long)NZ * NXP;
    const int nshot = geo->nshot, nrec = geo->nrec, nt = g->nt;
    // carve the scratch: c, bpad, fields [2][nshot][P], gz, gx, offsets, status
    float *p = base;
    float *c = p; p += al(P);
    float *bpad = p; p += al(P);
    float *fa = p; p += al(P * nshot);
    float *fb = p; p += al(P * nshot);
    float *gz = p; p += al(NZ);
    float *gx = p; p += al(NXP);
    int *offs = reinterpret_cast<int *>(p);
    int *status = offs + nshot + nrec;

    // offsets and a cleared status word (host -> scratch), model preparation with its check, and the
    // status back; h and st_h are locals, so the call waits for the stream before it uses them again
    std::vector<int> h(nshot + nrec + 1, 0);
    for (int s = 0; s < nshot; ++s) h[s] = (geo->src_iz[s] + o) * NXP + geo->src_ix[s] + o;
    for (int r = 0; r < nrec; ++r) h[nshot + r] = (geo->rec_iz[r] + o) * NXP + geo->rec_ix[r] + o;
#define CKS(call)                                                                                    \
    do {                                                                                             \
        cudaError_t e_ = (call);                                                                     \
        if (e_ != cudaSuccess) {                                                                     \
            snprintf(g_err, sizeof(g_err), "fwime_forward_static: %s: %s", #call, cudaGetErrorString(e_)); \
            return FWIME_ECUDA;                                                                      \
        }                                                                                            \
    } while (0)
    CKS(cudaMemcpyAsync(offs, h.data(), h.size() * sizeof(int), cudaMemcpyHostToDevice, st));
    PrepArgs pa{};
    pa.nz = g->nz; pa.nx = g->nx; pa.o = o; pa.NZ = NZ; pa.NX = NX; pa.NXP = NXP; pa.W = g->sponge; pa.dt = g->dt;
    pa.cfl_limit2 = cfl_vmax2(g->dt, g->dx, g->dz);
    pa.v = v; pa.c = c; pa.gz = gz; pa.gx = gx; pa.bpad = bpad; pa.status = status;
    CKS(launch_prep(pa, st));
    int st_h = 0;
    CKS(cudaMemcpyAsync(&st_h, status, sizeof(int), cudaMemcpyDeviceToHost, st));
    CKS(cudaStreamSynchronize(st));
    if (st_h & ST_CFL) {
        snprintf(g_err, sizeof(g_err),
                 "fwime_forward_static: velocity violates the CFL bound (vmax < %.6g m/s) or is not positive",
                 std::sqrt((double)pa.cfl_limit2));
        return FWIME_ECFL;
    }
    CKS(cudaMemsetAsync(fa, 0, sizeof(float) * P * nshot, st));
    CKS(cudaMemsetAsync(fb, 0, sizeof(float) * P * nshot, st));
    CKS(cudaMemsetAsync(d, 0, sizeof(float) * (size_t)nshot * nt * nrec, st));

    PropArgs a;
    std::memset(&a, 0, sizeof(a));
    a.NZ = NZ; a.NXP = NXP; a.P = P;
    a.nstrip = (NXP + STRIP - 1) / STRIP;
    const int rows = NZ - 8;
    long long nct = std::max<long long>(1, (152LL * 32 + (long long)a.nstrip * nshot - 1) / ((long long)a.nstrip * nshot));
    int zc = (int)((rows + nct - 1) / nct);
    a.zchunk = std::min(std::max(zc, 8), 256);
    a.nchunk = (rows + a.zchunk - 1) / a.zchunk;
    const double A8[5] = {-205.0 / 72.0, 8.0 / 5.0, -1.0 / 5.0, 8.0 / 315.0, -1.0 / 560.0};
    for (int k = 0; k < 5; ++k) {
        a.ax[k] = (float)(A8[k] / ((double)g->dx * g->dx));
        a.az[k] = (float)(A8[k] / ((double)g->dz * g->dz));
    }
    a.inv_dt2 = (float)(1.0 / ((double)g->dt * g->dt));
    a.src_scale = (float)(1.0 / ((double)g->dx * g->dz));
    a.c = c; a.gz = gz; a.gx = gx;
    a.zs_lo = o; a.zs_hi = o + g->nz;
    a.src_off = offs;
    a.src_stride = nt;
    PointsArgs r{};
    r.nrec = nrec; r.P = P; r.rec_off = offs + nshot; r.dstride = (long long)nt * nrec;
    float *curf = fa, *prvf = fb;
    for (int n = 0; n + 1 < nt; ++n) {
        a.cur = curf; a.prev = prvf; a.out = prvf; a.src_amp = w + n;
        CKS(launch_prop(a, nshot, st));
        r.f1 = prvf; r.d = d + (size_t)(n + 1) * nrec;
        CKS(launch_points(r, nshot, st));
        std::swap(curf, prvf);
    }
#undef CKS
    return FWIME_OK;
}

extern "C" int fwime_static_last_error(char *buf, size_t n)
{
    if (!buf || n == 0) return FWIME_EINVAL;
    snprintf(buf, n, "%s", g_err);
    return FWIME_OK;
}
