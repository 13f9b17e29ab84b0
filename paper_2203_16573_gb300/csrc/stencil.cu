// stencil.cu -- staggered-grid leapfrog step of the acoustic system and its
// exact transpose, with line injection / sampling fused in (sm_103a).
//
// Forward step n (eqn:awepm discretised as in "Synthetic models and
// simulation"; staggered grid, order 2 in time, 2k in space):
//   v^{n+1/2} = A_v v^{n-1/2} - B_v dt/(rho h) D+ p^n        (+ f[n] on z_s)
//   p^{n+1}   = A_p p^n - B_p kappa dt/h D- v^{n+1/2}          (+ h[n] on z_s)
//   traces n: P p^{n+1}, P v_z^{n+1/2}      (linear interpolation in depth)
// A = (1-s)/(1+s), B = 1/(1+s), s = (sigma_x + sigma_z) dt/2 (sponge).
// D+ u(j+1/2) = sum_m c_m (u[j+m] - u[j-m+1]);  D- w(i) = sum_m c_m (w[i+m-1] - w[i-m]);
// fields vanish outside the grid, so (D+)^T = -D- exactly.
//
// One CTA updates a TX x TZ tile in one launch: it stages p^n over the tile
// plus a 2k halo in shared memory, recomputes v^{n+1/2} over the tile plus a
// k halo (x halo for v_x, z halo for v_z) so that the p update needs no other
// CTA's output, and writes p, v_x, v_z of its own tile to the other buffer of
// a ping-pong pair. Per grid point and step that is 16 B read (p, v_x, v_z,
// kappa) and 12 B written; halo re-reads hit L2.
//
// The transposed step (Appendix A's adjoint state, run in reverse time)
// has the same shape with the coefficients moved inside the differences:
//   q = C_p pbar;  vbar' = vbar + D+ q;  pbar <- A_p pbar + D- (C_v vbar');  vbar <- A_v vbar'
// so one kernel of the same structure computes it exactly (FP32, identical
// coefficient arithmetic to the forward kernel).
#include "ssx_internal.cuh"

namespace ssx {

namespace {

__device__ __forceinline__ void damp(float s, float &A, float &B) {
    if (s == 0.0f) {
        A = 1.0f;
        B = 1.0f;
    } else {
        B = 1.0f / (1.0f + s);
        A = (1.0f - s) * B;
    }
}

__device__ __forceinline__ float row_weight(int k, int k0, float w0, float w1) {
    return (k == k0) ? w0 : ((k == k0 + 1) ? w1 : 0.0f);
}

constexpr int kThreads = 256;

template <int R, int TX, int TZ>
__global__ void __launch_bounds__(kThreads) k_fwd(const FwdArgs a) {
    constexpr int H = 2 * R;
    constexpr int PW = TX + 2 * H, PH = TZ + 2 * H;
    constexpr int VXW = TX + 2 * R - 1, VZH = TZ + 2 * R - 1;
    __shared__ float sp[PH][PW];
    __shared__ float svx[TZ][VXW];
    __shared__ float svz[VZH][TX];

    const GridArgs &g = a.g;
    const int pitch = g.pitch;
    const int i0 = blockIdx.x * TX, k0 = blockIdx.y * TZ;
    const int tid = threadIdx.x;

    // p^n over the tile and a 2k halo (the apron makes every read in bounds)
    for (int idx = tid; idx < PH * PW; idx += kThreads) {
        const int r = idx / PW, c = idx - r * PW;
        sp[r][c] = a.p_in[(k0 - H + r) * pitch + (i0 - H + c)];
    }
    __syncthreads();

    // v_x^{n+1/2} on the tile rows, columns i0-k .. i0+TX+k-2
    for (int idx = tid; idx < TZ * VXW; idx += kThreads) {
        const int r = idx / VXW, jj = idx - r * VXW;
        const int k = k0 + r, j = i0 - R + jj;
        float val = 0.0f;
        if (k < g.NZ && j >= 0 && j < g.NX - 1) {
            const float *row = &sp[r + H][jj + R];
            float d = 0.0f;
#pragma unroll
            for (int m = 1; m <= R; m++) d += g.c[m - 1] * (row[m] - row[1 - m]);
            float A, B;
            damp(g.sxh[j] + g.szi[k], A, B);
            const int o = k * pitch + j;
            val = A * a.vx_in[o] - (B * g.cv) * d;
            if (jj >= R && jj < R + TX) a.vx_out[o] = val;
        }
        svx[r][jj] = val;
    }
    // v_z^{n+1/2} on rows k0-k .. k0+TZ+k-2, the tile columns
    for (int idx = tid; idx < VZH * TX; idx += kThreads) {
        const int kk = idx / TX, c = idx - kk * TX;
        const int k = k0 - R + kk, i = i0 + c;
        float val = 0.0f;
        if (i < g.NX && k >= 0 && k < g.NZ - 1) {
            float d = 0.0f;
#pragma unroll
            for (int m = 1; m <= R; m++)
                d += g.c[m - 1] * (sp[kk + R + m][c + H] - sp[kk + R + 1 - m][c + H]);
            float A, B;
            damp(g.sxi[i] + g.szh[k], A, B);
            const int o = k * pitch + i;
            const float cvz = B * g.cv;
            val = A * a.vz_in[o] - cvz * d;
            if (a.fsrc) {   // vertical load f e_z delta(z - z_s)
                const float w = row_weight(k, a.src.kv, a.src.wv0, a.src.wv1);
                const int jl = i - a.src.i0;
                if (w != 0.0f && jl >= 0 && jl < a.src.n)
                    val += cvz * (w * a.src.scale) * (float)a.fsrc[(size_t)a.n * a.src.n + jl];
            }
            if (kk >= R && kk < R + TZ) {
                a.vz_out[o] = val;
                if (a.outv) {
                    const float w = row_weight(k, a.rec.kv, a.rec.wv0, a.rec.wv1);
                    const int jl = i - a.rec.i0;
                    if (w != 0.0f && jl >= 0 && jl < a.rec.n)
                        atomicAdd(&a.outv[(size_t)a.n * a.rec.n + jl], (double)w * (double)val);
                }
            }
        }
        svz[kk][c] = val;
    }
    __syncthreads();

    // p^{n+1} on the tile
    for (int idx = tid; idx < TZ * TX; idx += kThreads) {
        const int r = idx / TX, c = idx - r * TX;
        const int k = k0 + r, i = i0 + c;
        if (k < g.NZ && i < g.NX) {
            float d = 0.0f;
#pragma unroll
            for (int m = 1; m <= R; m++) {
                d += g.c[m - 1] * (svx[r][c + R + m - 1] - svx[r][c + R - m]);
                d += g.c[m - 1] * (svz[r + R + m - 1][c] - svz[r + R - m][c]);
            }
            float A, B;
            damp(g.sxi[i] + g.szi[k], A, B);
            const int o = k * pitch + i;
            const float cp = B * g.kap[o];
            float val = A * sp[r + H][c + H] - cp * d;
            if (a.hsrc) {   // constitutive defect h delta(z - z_s)
                const float w = row_weight(k, a.src.kp, a.src.wp0, a.src.wp1);
                const int jl = i - a.src.i0;
                if (w != 0.0f && jl >= 0 && jl < a.src.n)
                    val += cp * (w * a.src.scale) * (float)a.hsrc[(size_t)a.n * a.src.n + jl];
            }
            a.p_out[o] = val;
            if (a.outp) {
                const float w = row_weight(k, a.rec.kp, a.rec.wp0, a.rec.wp1);
                const int jl = i - a.rec.i0;
                if (w != 0.0f && jl >= 0 && jl < a.rec.n)
                    atomicAdd(&a.outp[(size_t)a.n * a.rec.n + jl], (double)w * (double)val);
            }
        }
    }
}

template <int R, int TX, int TZ>
__global__ void __launch_bounds__(kThreads) k_adj(const AdjArgs a) {
    constexpr int H = 2 * R;
    constexpr int PW = TX + 2 * H, PH = TZ + 2 * H;
    constexpr int VXW = TX + 2 * R - 1, VZH = TZ + 2 * R - 1;
    __shared__ float sq[PH][PW];
    __shared__ float svx[TZ][VXW];
    __shared__ float svz[VZH][TX];

    const GridArgs &g = a.g;
    const int pitch = g.pitch;
    const int i0 = blockIdx.x * TX, k0 = blockIdx.y * TZ;
    const int tid = threadIdx.x;

    // q = C_p pbar over tile + 2k halo; read out the transposed p injection
    for (int idx = tid; idx < PH * PW; idx += kThreads) {
        const int r = idx / PW, c = idx - r * PW;
        const int k = k0 - H + r, i = i0 - H + c;
        float q = 0.0f;
        if (k >= 0 && k < g.NZ && i >= 0 && i < g.NX) {
            float A, B;
            damp(g.sxi[i] + g.szi[k], A, B);
            const int o = k * pitch + i;
            q = (B * g.kap[o]) * a.p_in[o];
            if (a.hbar && r >= H && r < H + TZ && c >= H && c < H + TX) {
                const float w = row_weight(k, a.src.kp, a.src.wp0, a.src.wp1);
                const int jl = i - a.src.i0;
                if (w != 0.0f && jl >= 0 && jl < a.src.n)
                    atomicAdd(&a.hbar[(size_t)a.n * a.src.n + jl],
                              (double)(w * a.src.scale) * (double)q);
            }
        }
        sq[r][c] = q;
    }
    __syncthreads();

    // vbar_x' = vbar_x + D+ q; keep C_vx vbar_x' for the p update
    for (int idx = tid; idx < TZ * VXW; idx += kThreads) {
        const int r = idx / VXW, jj = idx - r * VXW;
        const int k = k0 + r, j = i0 - R + jj;
        float val = 0.0f;
        if (k < g.NZ && j >= 0 && j < g.NX - 1) {
            const float *row = &sq[r + H][jj + R];
            float d = 0.0f;
#pragma unroll
            for (int m = 1; m <= R; m++) d += g.c[m - 1] * (row[m] - row[1 - m]);
            float A, B;
            damp(g.sxh[j] + g.szi[k], A, B);
            const int o = k * pitch + j;
            const float vb = a.vx_in[o] + d;
            val = (B * g.cv) * vb;
            if (jj >= R && jj < R + TX) a.vx_out[o] = A * vb;
        }
        svx[r][jj] = val;
    }
    // vbar_z' likewise; read out the transposed velocity injection
    for (int idx = tid; idx < VZH * TX; idx += kThreads) {
        const int kk = idx / TX, c = idx - kk * TX;
        const int k = k0 - R + kk, i = i0 + c;
        float val = 0.0f;
        if (i < g.NX && k >= 0 && k < g.NZ - 1) {
            float d = 0.0f;
#pragma unroll
            for (int m = 1; m <= R; m++)
                d += g.c[m - 1] * (sq[kk + R + m][c + H] - sq[kk + R + 1 - m][c + H]);
            float A, B;
            damp(g.sxi[i] + g.szh[k], A, B);
            const int o = k * pitch + i;
            const float vb = a.vz_in[o] + d;
            val = (B * g.cv) * vb;
            if (kk >= R && kk < R + TZ) {
                if (a.fbar) {
                    const float w = row_weight(k, a.src.kv, a.src.wv0, a.src.wv1);
                    const int jl = i - a.src.i0;
                    if (w != 0.0f && jl >= 0 && jl < a.src.n)
                        atomicAdd(&a.fbar[(size_t)a.n * a.src.n + jl],
                                  (double)(w * a.src.scale) * (double)val);
                }
                float out = A * vb;
                if (a.yv && a.n >= 1) {   // transposed sampling of step n-1
                    const float w = row_weight(k, a.rec.kv, a.rec.wv0, a.rec.wv1);
                    const int jl = i - a.rec.i0;
                    if (w != 0.0f && jl >= 0 && jl < a.rec.n)
                        out += w * (float)a.yv[(size_t)(a.n - 1) * a.rec.n + jl];
                }
                a.vz_out[o] = out;
            }
        }
        svz[kk][c] = val;
    }
    __syncthreads();

    // pbar <- A_p pbar + D- (C_v vbar')
    for (int idx = tid; idx < TZ * TX; idx += kThreads) {
        const int r = idx / TX, c = idx - r * TX;
        const int k = k0 + r, i = i0 + c;
        if (k < g.NZ && i < g.NX) {
            float d = 0.0f;
#pragma unroll
            for (int m = 1; m <= R; m++) {
                d += g.c[m - 1] * (svx[r][c + R + m - 1] - svx[r][c + R - m]);
                d += g.c[m - 1] * (svz[r + R + m - 1][c] - svz[r + R - m][c]);
            }
            float A, B;
            damp(g.sxi[i] + g.szi[k], A, B);
            const int o = k * pitch + i;
            float out = A * a.p_in[o] + d;
            if (a.yp && a.n >= 1) {
                const float w = row_weight(k, a.rec.kp, a.rec.wp0, a.rec.wp1);
                const int jl = i - a.rec.i0;
                if (w != 0.0f && jl >= 0 && jl < a.rec.n)
                    out += w * (float)a.yp[(size_t)(a.n - 1) * a.rec.n + jl];
            }
            a.p_out[o] = out;
        }
    }
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

constexpr int kTX = 64, kTZ = 16;
static_assert(kTX <= TILE_X_MAX && kTZ <= TILE_Z_MAX, "tile larger than the allocation rounding");

}  // namespace

void tile_shape(int R, int *tx, int *tz) {
    (void)R;
    *tx = kTX;
    *tz = kTZ;
}

cudaError_t launch_fwd_step(const FwdArgs &a, int R, cudaStream_t s) {
    dim3 grid((a.g.NX + kTX - 1) / kTX, (a.g.NZ + kTZ - 1) / kTZ);
    switch (R) {
        case 1: k_fwd<1, kTX, kTZ><<<grid, kThreads, 0, s>>>(a); break;
        case 2: k_fwd<2, kTX, kTZ><<<grid, kThreads, 0, s>>>(a); break;
        case 3: k_fwd<3, kTX, kTZ><<<grid, kThreads, 0, s>>>(a); break;
        case 4: k_fwd<4, kTX, kTZ><<<grid, kThreads, 0, s>>>(a); break;
        default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

cudaError_t launch_adj_step(const AdjArgs &a, int R, cudaStream_t s) {
    dim3 grid((a.g.NX + kTX - 1) / kTX, (a.g.NZ + kTZ - 1) / kTZ);
    switch (R) {
        case 1: k_adj<1, kTX, kTZ><<<grid, kThreads, 0, s>>>(a); break;
        case 2: k_adj<2, kTX, kTZ><<<grid, kThreads, 0, s>>>(a); break;
        case 3: k_adj<3, kTX, kTZ><<<grid, kThreads, 0, s>>>(a); break;
        case 4: k_adj<4, kTX, kTZ><<<grid, kThreads, 0, s>>>(a); break;
        default: return cudaErrorInvalidValue;
    }
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
