// noalloc.cu -- forward modelling d = S h for callers that cannot allocate
// device memory.
//
// Some hosts of this library may not call cudaMalloc at all: code running
// inside a framework that owns the whole device pool, a plugin whose memory
// budget is fixed up front, or a caller that must not trigger an allocation
// (and the implicit synchronisation it may bring) in the middle of its own
// work. ssx_forward_noalloc serves them: the caller passes the inputs and the
// output buffer, and every piece of scratch the sweep needs -- the padded
// kappa field, the two ping-pong wavefield triples, the sponge tables and the
// model maximum -- lives in one file-scope device array of fixed size. The
// array is reserved on a GPU when the library's module is first used there
// (with CUDA's lazy module loading that may be inside the first call) and is
// held by that GPU until the process exits. No cudaMalloc, cudaFree, graph
// instantiation or other allocating call is made.
//
// The array is shared by every call on a device: its contents are the last
// call's, so each call clears what must start at zero, and calls whose work
// overlaps on the GPU (different streams, or different threads) race on it.
#include <cuda_runtime.h>

#include <cmath>
#include <mutex>

#include "../../include/ssx.h"
#include "ssx_internal.cuh"

using namespace ssx;

namespace {

// Scratch capacity in floats (16 MiB): enough for a padded grid of about
// 590 000 storage points (e.g. the 681 x 381 padded 601 x 301 model).
constexpr size_t kScratchFloats = SSX_NOALLOC_MAX_FLOATS;

static __device__ __align__(256) float g_scratch[kScratchFloats];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
float *g_scratch_ptr[kMaxDevices] = {};   // device address of g_scratch, per device

// Host code may not pass g_scratch itself to a kernel: in host code that name
// is a host-side stand-in, not a device address. Its device address is looked
// up once per device, with that device current.
int scratch_address(float **out) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return SSX_ERR_CUDA;
    std::lock_guard<std::mutex> lock(g_mu);
    if (!g_scratch_ptr[dev]) {
        void *p = nullptr;
        if (cudaGetSymbolAddress(&p, g_scratch) != cudaSuccess || !p) return SSX_ERR_CUDA;
        g_scratch_ptr[dev] = (float *)p;
    }
    *out = g_scratch_ptr[dev];
    return SSX_OK;
}

}  // namespace

extern "C" int ssx_forward_noalloc(const ssx_grid_desc *gd, const ssx_geom_desc *gm,
                                   const float *v_dev, double rho, const double *h_dev,
                                   double *d_dev, void *stream) {
    if (!gd || !gm || !v_dev || !h_dev || !d_dev || !(rho > 0)) return SSX_ERR_ARG;
    if (gd->nx < 8 || gd->nz < 8 || gd->nt < 1 || !(gd->h > 0) || !(gd->dt > 0) ||
        gd->n_sponge < 0 || gd->space_order < 2 || gd->space_order > 8 || gd->space_order % 2)
        return SSX_ERR_ARG;
    const int R = gd->space_order / 2, nsp = gd->n_sponge;
    // the padded grid alone must fit the scratch: checked in 64-bit arithmetic
    // before any int layout arithmetic can overflow
    const long long NXl = (long long)gd->nx + 2LL * nsp, NZl = (long long)gd->nz + 2LL * nsp;
    if (NXl * NZl > (long long)kScratchFloats) return SSX_ERR_ARG;
    const FieldLayout L = field_layout((int)NXl, (int)NZl);
    const size_t E = L.elems();
    const size_t tab = 2 * (size_t)(L.NX + L.NZ);
    const size_t need = 7 * E + tab + 64;
    if (need > kScratchFloats) return SSX_ERR_ARG;   // grid larger than the fixed scratch
    Line src{}, rec{};
    if (line_at(gm->z_s / gd->h + nsp, L.NZ, gd->nx, nsp, gm->ix_line0, gm->n_line, 1.0, &src) ||
        line_at(gm->z_r / gd->h + nsp, L.NZ, gd->nx, nsp, gm->ix_rec0, gm->n_rec, 1.0, &rec))
        return SSX_ERR_ARG;

    float *base = nullptr;
    int rc = scratch_address(&base);
    if (rc != SSX_OK) return rc;
    cudaStream_t s = (cudaStream_t)stream;
    float *kap_mem = base;                 // kap | buffer 0 | buffer 1 | tables | vmax
    float *tabs = base + 7 * E;
    float *vmax = tabs + tab;
    const size_t nv = (size_t)gd->nx * gd->nz;

    // the array keeps the previous call's contents: clear fields and apron
    if (cudaMemsetAsync(base, 0, 7 * E * sizeof(float), s) != cudaSuccess) return SSX_ERR_CUDA;
    if (cudaMemsetAsync(d_dev, 0, (size_t)gd->nt * gm->n_rec * sizeof(double), s) != cudaSuccess)
        return SSX_ERR_CUDA;
    if (launch_vmax(v_dev, (int)nv, vmax, s) != cudaSuccess) return SSX_ERR_CUDA;
    // CFL bound v_max dt/h sqrt(2) sum |c_m| < 1 (one 4-byte read, synchronising)
    float vm = 0.f;
    if (cudaMemcpyAsync(&vm, vmax, sizeof(float), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess)
        return SSX_ERR_CUDA;
    if (!(vm > 0) || !std::isfinite(vm)) return SSX_ERR_ARG;
    if (!(vm * gd->dt / gd->h * std::sqrt(2.0) * kWeightsAbsSum[R] < 1.0)) return SSX_ERR_CFL;

    float *kap = kap_mem + L.origin();
    if (launch_fill_kappa(kap, L, v_dev, gd->nx, gd->nz, nsp, 0, rho, gd->dt / gd->h, s) !=
        cudaSuccess)
        return SSX_ERR_CUDA;
    // the sponge tables of a context's grid: same scale from the same maximum
    const double sdt = sponge_scale(vm, nsp, gd->h, gd->dt);
    if (launch_sponge_table(tabs, tabs + L.NX, L.NX, gd->nx, nsp, sdt, s) != cudaSuccess ||
        launch_sponge_table(tabs + 2 * L.NX, tabs + 2 * L.NX + L.NZ, L.NZ, gd->nz, nsp, sdt, s) !=
            cudaSuccess)
        return SSX_ERR_CUDA;

    FwdArgs a{};
    GridArgs &g = a.g;
    g.NX = L.NX;
    g.NZ = L.NZ;
    g.pitch = L.pitch;
    g.kap = kap;
    g.sxi = tabs;
    g.sxh = tabs + L.NX;
    g.szi = tabs + 2 * L.NX;
    g.szh = tabs + 2 * L.NX + L.NZ;
    g.cv = (float)(gd->dt / (rho * gd->h));
    for (int m = 0; m < kMaxR; m++) g.c[m] = kWeights[R][m];
    g.in_x0 = nsp;
    g.in_x1 = nsp + gd->nx - 1;
    g.in_z0 = nsp;
    g.in_z1 = nsp + gd->nz - 1;
    a.src = src;
    a.hsrc = h_dev;
    a.fsrc = nullptr;
    a.rec = rec;
    a.outp = d_dev;
    a.outv = nullptr;
    float *f[2][3];
    for (int b = 0; b < 2; b++)
        for (int k = 0; k < 3; k++) f[b][k] = kap_mem + (1 + 3 * b + k) * E + L.origin();
    for (int n = 0; n < gd->nt; n++) {
        const int bi = n & 1, bo = bi ^ 1;
        a.p_in = f[bi][0];
        a.vx_in = f[bi][1];
        a.vz_in = f[bi][2];
        a.p_out = f[bo][0];
        a.vx_out = f[bo][1];
        a.vz_out = f[bo][2];
        a.n = n;
        if (launch_fwd_step(a, R, 0, s, false) != cudaSuccess) return SSX_ERR_CUDA;
    }
    return SSX_OK;
}
