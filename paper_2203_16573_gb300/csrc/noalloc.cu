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
// model maximum -- lives in one file-scope device array of fixed size,
// reserved when the library's module is loaded on a GPU and held by that GPU
// until the process exits. No cudaMalloc, cudaFree, graph instantiation or
// other allocating call is made.
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

int row_of(double zeta, int *k, float *w0, float *w1) {
    const int kk = (int)std::floor(zeta + 1e-6);
    double f = zeta - kk;
    if (f < 1e-6) f = 0.0;
    *k = kk;
    *w0 = (float)(1.0 - f);
    *w1 = (float)f;
    return 0;
}

bool line_at(int NX, int NZ, int nx, int nsp, double h, double z, int ix0, int n, Line *L) {
    const double zeta = z / h + nsp;
    row_of(zeta, &L->kp, &L->wp0, &L->wp1);
    row_of(zeta - 0.5, &L->kv, &L->wv0, &L->wv1);
    if (!(L->kp >= 0 && L->kp + 1 < NZ && L->kv >= 0 && L->kv + 1 < NZ - 1)) return false;
    if (ix0 < 0 || n < 1 || ix0 + n > nx) return false;
    (void)NX;
    L->i0 = ix0 + nsp;
    L->n = n;
    L->scale = 1.0f;
    return true;
}

// sponge tables from the device-resident model maximum (no host round trip)
__global__ void k_sponge_from_vmax(float *ti, float *th, int N, int n_phys, int nsp, double h,
                                   double dt, const float *vmax) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N) return;
    const double smax = nsp > 0 ? 3.0 * (double)*vmax * log(1000.0) / (2.0 * nsp * h) : 0.0;
    for (int half = 0; half < 2; half++) {
        const double pos = i + 0.5 * half;
        const double d = fmax(0.0, fmax((double)nsp - pos, pos - (double)(nsp + n_phys - 1)));
        const double s = nsp > 0 ? 0.5 * dt * smax * (d / nsp) * (d / nsp) : 0.0;
        (half ? th : ti)[i] = (float)s;
    }
}

const float kW[5][kMaxR] = {
    {0.f, 0.f, 0.f, 0.f},
    {1.0f, 0.f, 0.f, 0.f},
    {9.0f / 8.0f, -1.0f / 24.0f, 0.f, 0.f},
    {75.0f / 64.0f, -25.0f / 384.0f, 3.0f / 640.0f, 0.f},
    {1225.0f / 1024.0f, -245.0f / 3072.0f, 49.0f / 5120.0f, -5.0f / 7168.0f},
};

int round_up_i(int a, int b) { return (a + b - 1) / b * b; }

}  // namespace

extern "C" int ssx_forward_noalloc(const ssx_grid_desc *gd, const ssx_geom_desc *gm,
                                   const float *v_dev, double rho, const double *h_dev,
                                   double *d_dev, void *stream) {
    if (!gd || !gm || !v_dev || !h_dev || !d_dev || !(rho > 0)) return SSX_ERR_ARG;
    if (gd->nx < 8 || gd->nz < 8 || gd->nt < 1 || !(gd->h > 0) || !(gd->dt > 0) ||
        gd->n_sponge < 0 || gd->space_order < 2 || gd->space_order > 8 || gd->space_order % 2)
        return SSX_ERR_ARG;
    const int R = gd->space_order / 2, nsp = gd->n_sponge;
    FieldLayout L{};
    L.NX = gd->nx + 2 * nsp;
    L.NZ = gd->nz + 2 * nsp;
    L.pitch = round_up_i(round_up_i(L.NX, TILE_X_MAX) + 2 * GX, 32);
    L.rows = round_up_i(L.NZ, TILE_Z_MAX) + 2 * GZ;
    const size_t E = L.elems();
    const size_t tab = 2 * (size_t)(L.NX + L.NZ);
    const size_t need = 7 * E + tab + 64;
    if (need > kScratchFloats) return SSX_ERR_ARG;   // grid larger than the fixed scratch
    Line src{}, rec{};
    if (!line_at(L.NX, L.NZ, gd->nx, nsp, gd->h, gm->z_s, gm->ix_line0, gm->n_line, &src) ||
        !line_at(L.NX, L.NZ, gd->nx, nsp, gd->h, gm->z_r, gm->ix_rec0, gm->n_rec, &rec))
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
    double asum = 0.0;
    for (int m = 0; m < R; m++) asum += std::fabs((double)kW[R][m]);
    if (!(vm > 0) || !std::isfinite(vm)) return SSX_ERR_ARG;
    if (!(vm * gd->dt / gd->h * std::sqrt(2.0) * asum < 1.0)) return SSX_ERR_CFL;

    float *kap = kap_mem + L.origin();
    if (launch_fill_kappa(kap, L, v_dev, gd->nx, gd->nz, nsp, 0, rho, gd->dt / gd->h, s) !=
        cudaSuccess)
        return SSX_ERR_CUDA;
    k_sponge_from_vmax<<<(L.NX + 127) / 128, 128, 0, s>>>(tabs, tabs + L.NX, L.NX, gd->nx, nsp,
                                                          gd->h, gd->dt, vmax);
    k_sponge_from_vmax<<<(L.NZ + 127) / 128, 128, 0, s>>>(tabs + 2 * L.NX,
                                                          tabs + 2 * L.NX + L.NZ, L.NZ, gd->nz,
                                                          nsp, gd->h, gd->dt, vmax);
    if (cudaGetLastError() != cudaSuccess) return SSX_ERR_CUDA;

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
    for (int m = 0; m < kMaxR; m++) g.c[m] = kW[R][m];
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
