// stencil.cu -- set-up kernels of a grid (kappa dt/h, sponge tables, model
// maximum), the adjoint sweep's initial injection, and the dispatch of the
// step kernels (stencil_impl.cuh, instantiated per half order R in
// stencil_r<R>.cu) over R and the tile configurations.
#include <cmath>

#include "stencil_impl.cuh"

namespace ssx {

namespace {

// C_p = B_p kappa~ at every storage point, with B_p the pressure points'
// sponge factor (the same damp() as the steps) and 0 outside the padded grid,
// so the transposed step stages q = C_p pbar with one product and no tests.
__global__ void k_fill_cpk(float *cpk, const GridArgs a, int rows, int gz, int gx) {
    const int x = blockIdx.x * blockDim.x + threadIdx.x, y = blockIdx.y;
    if (x >= a.pitch || y >= rows) return;
    const int k = y - gz, i = x - gx;
    float v = 0.0f;
    if (k >= 0 && k < a.NZ && i >= 0 && i < a.NX) {
        float A, B;
        damp(a.sxi[i] + a.szi[k], A, B);
        v = __fmul_rn(B, a.kap[k * a.pitch + i]);
    }
    cpk[(size_t)y * a.pitch + x] = v;
}

// Adjoint state entering reverse step nt-1: the transposed sampling of the
// last trace sample, on zeroed fields (one thread per receiver column, so the
// two interpolation rows of a column never race).
__global__ void k_adj_init(const AdjArgs a, int nt) {
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= a.rec.n) return;
    const int i = a.rec.i0 + j;
    const int pitch = a.g.pitch;
    float *p = const_cast<float *>(a.p_in);
    float *vz = const_cast<float *>(a.vz_in);
    if (a.yp) {
        const float y = (float)a.yp[(size_t)(nt - 1) * a.rec.n + j];
        p[a.rec.kp * pitch + i] += a.rec.wp0 * y;
        if (a.rec.wp1 != 0.0f) p[(a.rec.kp + 1) * pitch + i] += a.rec.wp1 * y;
    }
    if (a.yv) {
        const float y = (float)a.yv[(size_t)(nt - 1) * a.rec.n + j];
        vz[a.rec.kv * pitch + i] += a.rec.wv0 * y;
        if (a.rec.wv1 != 0.0f) vz[(a.rec.kv + 1) * pitch + i] += a.rec.wv1 * y;
    }
}

// kappa dt/h on the padded grid; the model row of padded row k is
// clamp(row0 + clamp(k - nsp, 0, nz_grid-1), 0, nz_model-1) (edge replication
// into the sponge, and for a slab, of the slab's own edge rows).
__global__ void k_fill_kappa(float *kap, int NX, int NZ, int pitch, const float *vel, int nx,
                             int nz_model, int nz_grid, int nsp, int row0, double rho,
                             double dt_over_h) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const int k = blockIdx.y;
    if (i >= NX || k >= NZ) return;
    int ip = min(max(i - nsp, 0), nx - 1);
    int ks = min(max(k - nsp, 0), nz_grid - 1);
    int km = min(max(row0 + ks, 0), nz_model - 1);
    const double v = (double)vel[(size_t)km * nx + ip];
    kap[k * pitch + i] = (float)(rho * v * v * dt_over_h);
}

__global__ void k_sponge_table(float *ti, float *th, int N, int n_phys, int nsp, double smax_dt_half) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N) return;
    for (int half = 0; half < 2; half++) {
        const double pos = i + 0.5 * half;
        double d = fmax(0.0, fmax((double)nsp - pos, pos - (double)(nsp + n_phys - 1)));
        double s = nsp > 0 ? smax_dt_half * (d / nsp) * (d / nsp) : 0.0;
        (half ? th : ti)[i] = (float)s;
    }
}

__global__ void k_vmax(const float *v, int n, float *out) {
    __shared__ float red[1024];
    float m = 0.0f;
    for (int i = threadIdx.x; i < n; i += blockDim.x) m = fmaxf(m, v[i]);
    red[threadIdx.x] = m;
    __syncthreads();
    for (int s = blockDim.x / 2; s > 0; s >>= 1) {
        if (threadIdx.x < s) red[threadIdx.x] = fmaxf(red[threadIdx.x], red[threadIdx.x + s]);
        __syncthreads();
    }
    if (threadIdx.x == 0) *out = red[0];
}

}  // namespace

const float kWeights[5][kMaxR] = {
    {0.f, 0.f, 0.f, 0.f},
    {1.0f, 0.f, 0.f, 0.f},
    {9.0f / 8.0f, -1.0f / 24.0f, 0.f, 0.f},
    {75.0f / 64.0f, -25.0f / 384.0f, 3.0f / 640.0f, 0.f},
    {1225.0f / 1024.0f, -245.0f / 3072.0f, 49.0f / 5120.0f, -5.0f / 7168.0f},
};
const double kWeightsAbsSum[5] = {0.0, 1.0, 9.0 / 8 + 1.0 / 24,
                                  75.0 / 64 + 25.0 / 384 + 3.0 / 640,
                                  1225.0 / 1024 + 245.0 / 3072 + 49.0 / 5120 + 5.0 / 7168};

FieldLayout field_layout(int NX, int NZ) {
    auto up = [](int a, int b) { return (a + b - 1) / b * b; };
    FieldLayout L{};
    L.NX = NX;
    L.NZ = NZ;
    L.pitch = up(up(NX, TILE_X_MAX) + 2 * GX, 32);
    L.rows = up(NZ, TILE_Z_MAX) + 2 * GZ;
    return L;
}

void row_weights(double zeta, int *k, float *w0, float *w1) {
    const int kk = (int)std::floor(zeta + 1e-6);
    double f = zeta - kk;
    if (f < 1e-6) f = 0.0;
    *k = kk;
    *w0 = (float)(1.0 - f);
    *w1 = (float)f;
}

int line_at(double zeta, int NZ, int nx, int nsp, int ix0, int n, double scale, Line *out) {
    Line L{};
    row_weights(zeta, &L.kp, &L.wp0, &L.wp1);
    row_weights(zeta - 0.5, &L.kv, &L.wv0, &L.wv1);
    if (!(L.kp >= 0 && L.kp + 1 < NZ && L.kv >= 0 && L.kv + 1 < NZ - 1)) return 1;
    if (ix0 < 0 || n < 1 || ix0 > nx - n) return 2;
    L.i0 = ix0 + nsp;
    L.n = n;
    L.scale = (float)scale;
    *out = L;
    return 0;
}

double sponge_scale(double v_max, int nsp, double h, double dt) {
    const double smax = nsp > 0 ? 3.0 * v_max * std::log(1000.0) / (2.0 * nsp * h) : 0.0;
    return smax * dt * 0.5;
}

const TileCfg kTileCfgs[kNumTileCfgs] = {
#define SSX_CFG_ROW(id, TX, TZ, NT, V) {TX, TZ, NT, V},
    SSX_TILE_CONFIGS(SSX_CFG_ROW)
#undef SSX_CFG_ROW
};

#define SSX_BY_R(fn, ...)                                  \
    switch (R) {                                           \
        case 1: return fn##_r1(__VA_ARGS__);               \
        case 2: return fn##_r2(__VA_ARGS__);               \
        case 3: return fn##_r3(__VA_ARGS__);               \
        case 4: return fn##_r4(__VA_ARGS__);               \
    }

cudaError_t launch_fwd_step(const FwdArgs &a, int R, int cfg, cudaStream_t s, bool pdl) {
    SSX_BY_R(stencil_fwd_step, a, cfg, s, pdl)
    return cudaErrorInvalidValue;
}
cudaError_t launch_adj_step(const AdjArgs &a, int R, int cfg, cudaStream_t s, bool pdl) {
    SSX_BY_R(stencil_adj_step, a, cfg, s, pdl)
    return cudaErrorInvalidValue;
}
cudaError_t launch_fwd_persist(const FwdArgs &a, const PersistArgs &pa, int R, int cfg,
                               cudaStream_t s) {
    SSX_BY_R(stencil_fwd_persist, a, pa, cfg, s)
    return cudaErrorInvalidValue;
}
cudaError_t launch_adj_persist(const AdjArgs &a, const PersistArgs &pa, int R, int cfg,
                               cudaStream_t s) {
    SSX_BY_R(stencil_adj_persist, a, pa, cfg, s)
    return cudaErrorInvalidValue;
}
cudaError_t launch_multi(const JobSet &jobs, int total_tiles, int t, int R, int cfg,
                         cudaStream_t s, bool pdl) {
    SSX_BY_R(stencil_multi, jobs, total_tiles, t, cfg, s, pdl)
    return cudaErrorInvalidValue;
}
cudaError_t launch_multi_tab(const Job *jobs, int njobs, int total_tiles, int t, int R, int cfg,
                             cudaStream_t s, bool pdl) {
    SSX_BY_R(stencil_multi_tab, jobs, njobs, total_tiles, t, cfg, s, pdl)
    return cudaErrorInvalidValue;
}
int persist_capacity(int R, int cfg, bool adj) {
    SSX_BY_R(stencil_capacity, cfg, adj)
    return 0;
}
cudaError_t prepare_kernels() {
    cudaError_t e;
    if ((e = stencil_prepare_r1()) != cudaSuccess) return e;
    if ((e = stencil_prepare_r2()) != cudaSuccess) return e;
    if ((e = stencil_prepare_r3()) != cudaSuccess) return e;
    if ((e = stencil_prepare_r4()) != cudaSuccess) return e;
    if ((e = prepare_march_kernels()) != cudaSuccess) return e;
    if ((e = prepare_two_kernels()) != cudaSuccess) return e;
    return prepare_tma_kernels();
}

cudaError_t launch_fill_cpk(const GridArgs &a, const FieldLayout &L, float *cpk, cudaStream_t s) {
    dim3 grid((L.pitch + 127) / 128, L.rows);
    k_fill_cpk<<<grid, 128, 0, s>>>(cpk, a, L.rows, GZ, GX);
    return cudaGetLastError();
}

cudaError_t launch_adj_init(const AdjArgs &a, int nt, cudaStream_t s) {
    if (a.rec.n <= 0) return cudaSuccess;
    k_adj_init<<<(a.rec.n + 127) / 128, 128, 0, s>>>(a, nt);
    return cudaGetLastError();
}

cudaError_t launch_fill_kappa(float *kap, const FieldLayout &L, const float *vel, int nx, int nz,
                              int nsp, int row0, double rho, double dt_over_h, cudaStream_t s) {
    // nz: rows of the model array; the grid's own physical rows are NZ - 2 nsp
    dim3 grid((L.NX + 127) / 128, L.NZ);
    k_fill_kappa<<<grid, 128, 0, s>>>(kap, L.NX, L.NZ, L.pitch, vel, nx, nz, L.NZ - 2 * nsp,
                                      nsp, row0, rho, dt_over_h);
    return cudaGetLastError();
}

cudaError_t launch_sponge_table(float *ti, float *th, int N, int n_phys, int nsp,
                                double smax_dt_half, cudaStream_t s) {
    k_sponge_table<<<(N + 127) / 128, 128, 0, s>>>(ti, th, N, n_phys, nsp, smax_dt_half);
    return cudaGetLastError();
}

cudaError_t launch_vmax(const float *v, int n, float *out, cudaStream_t s) {
    k_vmax<<<1, 1024, 0, s>>>(v, n, out);
    return cudaGetLastError();
}

}  // namespace ssx
