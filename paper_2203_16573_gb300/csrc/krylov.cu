// krylov.cu -- FP64 vector kernels of Algorithm 1 (preconditioned CG) and of
// the diagonal operators (penalty A of eqn:penop, (I + alpha A^T A)^{-1/2} of
// eqn:defprecond).
//
// Inner products are deterministic: a fixed grid of kDotBlocks blocks, each
// reducing a fixed grid-stride slice with warp shuffles, then one block
// summing the partials in a fixed tree order. The PCG scalars (alpha_k,
// beta_k, <g,r>, <p,q>, ||r||^2) stay in device memory; kernels read them
// from there, so an iteration needs no host round trip except the 56-byte
// read of the scalar slots that decides the stop.
#include "ssx_internal.cuh"

namespace ssx {

namespace {

constexpr int kDotThreads = 256;

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    return v;
}

__device__ __forceinline__ void block_store_sum(double v, double *dst) {
    __shared__ double ws[kDotThreads / 32];
    v = warp_sum(v);
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    if (lane == 0) ws[wid] = v;
    __syncthreads();
    if (wid == 0) {
        v = lane < kDotThreads / 32 ? ws[lane] : 0.0;
        v = warp_sum(v);
        if (lane == 0) *dst = v;
    }
}

__global__ void __launch_bounds__(kDotThreads) k_dot_partial(const double *a, const double *b,
                                                             size_t n, double *partials) {
    double s = 0.0;
    for (size_t i = (size_t)blockIdx.x * kDotThreads + threadIdx.x; i < n;
         i += (size_t)kDotBlocks * kDotThreads)
        s = fma(a[i], b[i], s);
    block_store_sum(s, &partials[blockIdx.x]);
}

__global__ void __launch_bounds__(kDotBlocks) k_dot_finish(const double *partials, double *out) {
    __shared__ double red[kDotBlocks];
    red[threadIdx.x] = partials[threadIdx.x];
    __syncthreads();
    for (int s = kDotBlocks / 2; s > 0; s >>= 1) {
        if (threadIdx.x < s) red[threadIdx.x] += red[threadIdx.x + s];
        __syncthreads();
    }
    if (threadIdx.x == 0) *out = red[0];
}

// alpha_k = <g_k, r_k> / <p_k, q_k>; flag breakdown (non-positive or
// non-finite curvature) so the update kernel leaves h and r untouched.
__global__ void k_pcg_alpha(double *sc) {
    const double gr = sc[SC_GR], pq = sc[SC_PQ];
    const bool ok = (pq > 0.0) && (gr > 0.0) && isfinite(pq) && isfinite(gr);
    sc[SC_FLAG] = ok ? 0.0 : 1.0;
    sc[SC_ALPHA] = ok ? gr / pq : 0.0;
}

// h_{k+1} = h_k + alpha_k p_k;  r_{k+1} = r_k - alpha_k q_k;  partials of ||r_{k+1}||^2
__global__ void __launch_bounds__(kDotThreads) k_pcg_update(double *h, double *r, const double *p,
                                                            const double *q, size_t n,
                                                            const double *sc, double *partials) {
    const double al = sc[SC_ALPHA];
    const bool skip = sc[SC_FLAG] != 0.0;
    double s = 0.0;
    for (size_t i = (size_t)blockIdx.x * kDotThreads + threadIdx.x; i < n;
         i += (size_t)kDotBlocks * kDotThreads) {
        double ri = r[i];
        if (!skip) {
            h[i] = fma(al, p[i], h[i]);
            ri = fma(-al, q[i], ri);
            r[i] = ri;
        }
        s = fma(ri, ri, s);
    }
    block_store_sum(s, &partials[blockIdx.x]);
}

// beta_{k+1} = <g_{k+1}, r_{k+1}> / <g_k, r_k>
__global__ void k_pcg_beta(double *sc) {
    const double grn = sc[SC_GRNEW];
    sc[SC_BETA] = grn / sc[SC_GR];
    sc[SC_GR] = grn;
}

// p_{k+1} = g_{k+1} + beta_{k+1} p_k
__global__ void k_xpby(double *p, const double *g, size_t n, const double *sc) {
    const double be = sc[SC_BETA];
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (size_t)gridDim.x * blockDim.x)
        p[i] = fma(be, p[i], g[i]);
}

// out[t][c] = w[c] in[t][c]  (diagonal operators on a gather)
__global__ void k_colscale(double *out, const double *in, const double *w, int nt, int nc) {
    const size_t n = (size_t)nt * nc;
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (size_t)gridDim.x * blockDim.x)
        out[i] = w[i % nc] * in[i];
}

// q[t][c] += alpha w[c] in[t][c]
__global__ void k_colscale_add(double *q, const double *in, const double *w, double alpha, int nt,
                               int nc) {
    const size_t n = (size_t)nt * nc;
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (size_t)gridDim.x * blockDim.x)
        q[i] = fma(alpha * w[i % nc], in[i], q[i]);
}

int vec_blocks(size_t n) {
    size_t b = (n + 255) / 256;
    return (int)(b < 1216 ? (b < 1 ? 1 : b) : 1216);   // 8 x 152 SMs
}

}  // namespace

cudaError_t launch_dot(const double *a, const double *b, size_t n, double *partials, double *out,
                       cudaStream_t s) {
    k_dot_partial<<<kDotBlocks, kDotThreads, 0, s>>>(a, b, n, partials);
    k_dot_finish<<<1, kDotBlocks, 0, s>>>(partials, out);
    return cudaGetLastError();
}

cudaError_t launch_pcg_alpha(double *sc, cudaStream_t s) {
    k_pcg_alpha<<<1, 1, 0, s>>>(sc);
    return cudaGetLastError();
}

cudaError_t launch_pcg_update(double *h, double *r, const double *p, const double *q, size_t n,
                              double *sc, double *partials, cudaStream_t s) {
    k_pcg_update<<<kDotBlocks, kDotThreads, 0, s>>>(h, r, p, q, n, sc, partials);
    k_dot_finish<<<1, kDotBlocks, 0, s>>>(partials, sc + SC_RR);
    return cudaGetLastError();
}

cudaError_t launch_pcg_beta(double *sc, cudaStream_t s) {
    k_pcg_beta<<<1, 1, 0, s>>>(sc);
    return cudaGetLastError();
}

cudaError_t launch_xpby(double *p, const double *g, size_t n, const double *sc, cudaStream_t s) {
    k_xpby<<<vec_blocks(n), 256, 0, s>>>(p, g, n, sc);
    return cudaGetLastError();
}

cudaError_t launch_colscale(double *out, const double *in, const double *w, int nt, int nc,
                            cudaStream_t s) {
    k_colscale<<<vec_blocks((size_t)nt * nc), 256, 0, s>>>(out, in, w, nt, nc);
    return cudaGetLastError();
}

cudaError_t launch_colscale_add(double *q, const double *in, const double *w, double alpha,
                                int nt, int nc, cudaStream_t s) {
    k_colscale_add<<<vec_blocks((size_t)nt * nc), 256, 0, s>>>(q, in, w, alpha, nt, nc);
    return cudaGetLastError();
}

}  // namespace ssx
