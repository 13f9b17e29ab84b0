// gradient.cu -- kernels of the velocity gradient of the source subproblem's
// objective (the reduced objective of variable projection; eqn:esi and the
// paragraph after eqn:esis).
//
// With h fixed, Phi(c) = ||S[c] h - d||^2 depends on the model only through
// kappa (dt/h) in the pressure update p^{n+1} = A_p p^n + kappa~ B_p q^n,
// where q^n (minus the divergence of v^{n+1/2} plus the injected h) does not
// depend on kappa~. The discrete adjoint state method gives
//     dPhi/dkappa~ = sum_n pbar^{n+1} (p^{n+1} - A_p p^n) / kappa~,
// pbar^{n+1} = dPhi/dp^{n+1}, the adjoint pressure entering reverse step n of
// the transposed sweep driven by 2 (S h - d). kappa~ does not depend on n, so
// k_grad_accum adds one step of sum_n pbar^{n+1} (p^{n+1} - A_p p^n) (FP64,
// no division per step) and k_grad_fold divides by kappa~ once, mapping
// dPhi/dkappa~ on the padded grid to dPhi/dv on the physical model
// (kappa = rho v^2; the sponge copies the edge model values, so each edge
// point collects its copies).
#include "stencil_impl.cuh"

namespace ssx {
namespace {

// g[k][i] += pbar^{n+1} (p^{n+1} - A_p p^n) on the padded grid, FP64
__global__ void k_grad_accum(double *__restrict__ g, const float *__restrict__ mu,
                             const float *__restrict__ pn1, const float *__restrict__ pn,
                             const GridArgs a) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x, k = blockIdx.y;
    if (i >= a.NX || k >= a.NZ) return;
    const int o = k * a.pitch + i;
    float A, B;
    damp(__ldg(a.sxi + i) + __ldg(a.szi + k), A, B);
    const float inc = fmaf(-A, __ldcg(pn + o), __ldcg(pn1 + o));
    g[(size_t)k * a.NX + i] = fma((double)__ldcg(mu + o), (double)inc, g[(size_t)k * a.NX + i]);
}

// dPhi/dv[k][i] = 2 rho v (dt/h) sum of dPhi/dkappa~ = g / kappa~ over the
// padded points holding a copy of model point (k, i)
__global__ void k_grad_fold(double *__restrict__ out, const double *__restrict__ g,
                            const float *__restrict__ vel, const float *__restrict__ kap, int pitch,
                            int nx, int nz, int nsp, int NX, double scale) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x, k = blockIdx.y;
    if (i >= nx || k >= nz) return;
    const int K0 = k == 0 ? 0 : k + nsp, K1 = k == nz - 1 ? nz - 1 + 2 * nsp : k + nsp;
    const int I0 = i == 0 ? 0 : i + nsp, I1 = i == nx - 1 ? nx - 1 + 2 * nsp : i + nsp;
    double s = 0.0;
    for (int K = K0; K <= K1; K++)
        for (int I = I0; I <= I1; I++) s += g[(size_t)K * NX + I] / (double)__ldg(kap + K * pitch + I);
    out[(size_t)k * nx + i] = scale * (double)vel[(size_t)k * nx + i] * s;
}

// ybar = 2 (y - d): the derivative of ||y - d||^2 in the traces
__global__ void k_residual2(double *__restrict__ ybar, const double *__restrict__ y,
                            const double *__restrict__ d, size_t n) {
    for (size_t j = blockIdx.x * (size_t)blockDim.x + threadIdx.x; j < n;
         j += (size_t)gridDim.x * blockDim.x)
        ybar[j] = 2.0 * (y[j] - d[j]);
}

}  // namespace

cudaError_t launch_grad_accum(double *g, const float *mu, const float *pn1, const float *pn,
                              const GridArgs &a, cudaStream_t s) {
    dim3 grid((a.NX + 255) / 256, a.NZ);
    k_grad_accum<<<grid, 256, 0, s>>>(g, mu, pn1, pn, a);
    return cudaGetLastError();
}

cudaError_t launch_grad_fold(double *out, const double *g, const float *vel, const float *kap,
                             int pitch, int nx, int nz, int nsp, int NX, double scale,
                             cudaStream_t s) {
    dim3 grid((nx + 127) / 128, nz);
    k_grad_fold<<<grid, 128, 0, s>>>(out, g, vel, kap, pitch, nx, nz, nsp, NX, scale);
    return cudaGetLastError();
}

cudaError_t launch_residual2(double *ybar, const double *y, const double *d, size_t n,
                             cudaStream_t s) {
    k_residual2<<<1216, 256, 0, s>>>(ybar, y, d, n);
    return cudaGetLastError();
}

}  // namespace ssx
