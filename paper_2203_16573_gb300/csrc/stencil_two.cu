// stencil_two.cu -- temporal blocking: the phase kernel that advances a
// single sweep by two time steps per launch (spatial order 8).
//
// A step of the single-shot solve's slab phases is a short chain of
// dependent launches on a grid that lives in L2: each launch waits for the
// previous one, loads its tile's operands, computes and stores, and the
// chain's latency, not bandwidth, sets the time per step. This kernel takes
// two steps n, n+1 (forward) or n, n-1 (transposed, reverse time) in one
// launch. It loads p^n over the tile plus a 4k halo, v over the tile plus the
// reach of two steps and the constants, then
//   step A: v^{n+1/2} over the tile + 3k (each component in its own
//           direction) and p^{n+1} over the tile + 2k halo, kept in shared
//           memory (the halo points are the neighbours' points, recomputed);
//   step B: the ordinary step of the tile from those values, stored to the
//           sweep's other buffer.
// Launch t of a phase therefore reads buffer t mod 2 and writes the other
// one; a phase with an odd step count ends with a launch of one step.
// Injection acts on every point a step computes, sampling and the transposed
// read-outs on the tile's own points only (each trace sample still gets its
// two row contributions once). Every point's arithmetic is the strips'
// (fwd_strip / adj_strip) term for term, with the general sponge form, which
// is exact where the sponge factors are 1, so the results are identical bit
// for bit to one step per launch. Loads outside the padded grid read 0
// instead of the storage's zero apron (the 4k halo reaches beyond the apron).
#include "stencil_impl.cuh"

namespace ssx {
namespace {

constexpr int kR2 = 4;   // order 8

// A region [Z0, Z1) x [X0, X1) of points relative to the tile corner, stored
// row-major in shared memory with pitch X1 - X0.
template <int Z0, int Z1, int X0, int X1>
struct Reg {
    static constexpr int W = X1 - X0, NR = Z1 - Z0, N = W * NR;
    __device__ static __forceinline__ int at(int dk, int di) { return (dk - Z0) * W + (di - X0); }
    // f(dk, di) for every point, the points dealt out over the CTA's threads;
    // unrolled, so that a thread's points are independent chains in flight
    // together (their loads issued back to back)
    template <int NT, class F>
    __device__ static __forceinline__ void each(F &&f) {
#pragma unroll
        for (int q = 0; q < (N + NT - 1) / NT; q++) {
            const int e = (int)threadIdx.x + q * NT;
            if (N % NT == 0 || e < N) {
                const int r = e / W;
                f(Z0 + r, X0 + (e - r * W));
            }
        }
    }
};

// The regions of a two-step launch on a TX x TZ tile (H = 2k).
template <int TX, int TZ>
struct TwoRegs {
    static constexpr int R = kR2, H = 2 * R;
    using P0 = Reg<-2 * H, TZ + 2 * H, -2 * H, TX + 2 * H>;             // p^n (step A's input)
    using VX0 = Reg<-H, TZ + H, -H - R, TX + H + R - 1>;                 // v_x of step A
    using VZ0 = Reg<-H - R, TZ + H + R - 1, -H, TX + H>;                 // v_z of step A
    using P1 = Reg<-H, TZ + H, -H, TX + H>;                              // p^{n+1}; step B's input
    using VXB = Reg<0, TZ, -R, TX + R - 1>;                              // v_x of step B
    using VZB = Reg<-R, TZ + R - 1, 0, TX>;                              // v_z of step B
    using T = Reg<0, TZ, 0, TX>;                                         // the tile
};

__device__ __forceinline__ int clampi(int v, int lo, int hi) { return v < lo ? lo : (v > hi ? hi : v); }

// a field over the points of region RG into shared memory in the layout of
// region RL (which contains RG): points outside [0, nz) x [0, nx) of the
// padded grid read 0 (the storage holds 0 there)
template <class RG, class RL, int NT>
__device__ __forceinline__ void load_region(float *dst, const float *f, int pitch, int i0, int k0,
                                            int nx, int nz, bool cached) {
    RG::template each<NT>([&](int dk, int di) {
        const int k = k0 + dk, i = i0 + di;
        const bool in = k >= 0 && k < nz && i >= 0 && i < nx;
        dst[RL::at(dk, di)] = in ? (cached ? __ldg(f + k * pitch + i) : ldf(f + k * pitch + i)) : 0.0f;
    });
}

}  // namespace
}  // namespace ssx

namespace ssx {
namespace {

__device__ __forceinline__ bool in_tile(int dk, int di, int TX, int TZ) {
    return dk >= 0 && dk < TZ && di >= 0 && di < TX;
}

// The sponge profiles over the columns and rows of region P0 (sigma dt/2 at
// integer and half positions), staged once per launch: x tables at di + 2H,
// z tables at dk + 2H (indices clamped into the grid; masked points take any
// value).
template <int TX, int TZ>
struct Prof {
    static constexpr int H = 2 * kR2, PW = TX + 4 * H, PR = TZ + 4 * H, N = 2 * PW + 2 * PR;
    float v[N];
    __device__ __forceinline__ float xi(int di) const { return v[di + 2 * H]; }
    __device__ __forceinline__ float xh(int di) const { return v[PW + di + 2 * H]; }
    __device__ __forceinline__ float zi(int dk) const { return v[2 * PW + dk + 2 * H]; }
    __device__ __forceinline__ float zh(int dk) const { return v[2 * PW + PR + dk + 2 * H]; }
    template <int NT>
    __device__ __forceinline__ void load(const GridArgs &g, int i0, int k0) {
#pragma unroll
        for (int q = 0; q < (N + NT - 1) / NT; q++) {
            const int e = (int)threadIdx.x + q * NT;
            if (e < 2 * PW) {
                const int x = e < PW ? e : e - PW;
                const int i = clampi(i0 - 2 * H + x, 0, g.NX - 1);
                v[e] = __ldg((e < PW ? g.sxi : g.sxh) + i);
            } else if (e < N) {
                const int z = e - 2 * PW < PR ? e - 2 * PW : e - 2 * PW - PR;
                const int k = clampi(k0 - 2 * H + z, 0, g.NZ - 1);
                v[e] = __ldg((e - 2 * PW < PR ? g.szi : g.szh) + k);
            }
        }
    }
};

// One forward step n over regions: v_x on RX and v_z on RZ (into sVX, sVZ),
// then p on RP. Inputs: p^n on RIN (sP), the old v in the layouts RXI / RZI
// (sVXI, sVZI), kappa in the layout RK (sK). LAST: the tile's own points are
// stored to the sweep's output buffer; else p^{n+1} goes to sPO (layout RP).
// The tile's own points are sampled either way.
template <int TX, int TZ, int NT, class RX, class RZ, class RP, class RIN, class RXI, class RZI,
          class RK, bool LAST>
__device__ __forceinline__ void fwd_regions(const FwdArgs &a, const StepIO &io, int n, int i0, int k0,
                                            const Prof<TX, TZ> &pf, const float *sP, const float *sVXI, const float *sVZI,
                                            const float *sK, float *sVX, float *sVZ, float *sPO) {
    constexpr int R = kR2;
    const GridArgs &g = a.g;
    const int pitch = g.pitch, NX = g.NX, NZ = g.NZ;
    float cc[R];
#pragma unroll
    for (int m = 0; m < R; m++) cc[m] = g.c[m];
    const float cv = g.cv;
    // v_x^{n+1/2}
    RX::template each<NT>([&](int dk, int di) {
        const int k = k0 + dk, j = i0 + di;
        const bool ok = k >= 0 && k < NZ && j >= 0 && j < NX - 1;
        float d = 0.0f;
#pragma unroll
        for (int m = 1; m <= R; m++) d = fmaf(cc[m - 1], sP[RIN::at(dk, di + m)] - sP[RIN::at(dk, di + 1 - m)], d);
        float A, B;
        damp(pf.xh(di) + pf.zi(dk), A, B);
        float vx = fmaf(-(B * cv), d, A * sVXI[RXI::at(dk, di)]);
        vx = ok ? vx : 0.0f;
        sVX[RX::at(dk, di)] = vx;
        if (LAST && ok && in_tile(dk, di, TX, TZ)) st_out(io.vx_out + k * pitch + j, vx);
    });
    // v_z^{n+1/2}, with the vertical load f e_z delta(z - z_s) and the P v_z trace
    RZ::template each<NT>([&](int dk, int di) {
        const int kk = k0 + dk, i = i0 + di;
        const bool ok = i >= 0 && i < NX && kk >= 0 && kk < NZ - 1;
        float d = 0.0f;
#pragma unroll
        for (int m = 1; m <= R; m++) d = fmaf(cc[m - 1], sP[RIN::at(dk + m, di)] - sP[RIN::at(dk + 1 - m, di)], d);
        float A, B;
        damp(pf.xi(di) + pf.zh(dk), A, B);
        const float cvz = B * cv;
        float vz = fmaf(-cvz, d, A * sVZI[RZI::at(dk, di)]);
        if (a.fsrc && ok) {
            const float w = row_weight(kk, a.src.kv, a.src.wv0, a.src.wv1);
            const int js = i - a.src.i0;
            if (w != 0.0f && js >= 0 && js < a.src.n)
                vz = fmaf(cvz * (w * a.src.scale), (float)__ldcg(a.fsrc + (size_t)n * a.src.n + js), vz);
        }
        vz = ok ? vz : 0.0f;
        sVZ[RZ::at(dk, di)] = vz;
        if (ok && in_tile(dk, di, TX, TZ)) {
            if (LAST) st_out(io.vz_out + kk * pitch + i, vz);
            if (a.outv) {
                const float w = row_weight(kk, a.rec.kv, a.rec.wv0, a.rec.wv1);
                const int jr = i - a.rec.i0;
                if (w != 0.0f && jr >= 0 && jr < a.rec.n)
                    atomicAdd(&a.outv[(size_t)n * a.rec.n + jr], (double)w * (double)vz);
            }
        }
    });
    __syncthreads();
    // p^{n+1}, with the constitutive defect h delta(z - z_s) and the P p trace
    RP::template each<NT>([&](int dk, int di) {
        const int k = k0 + dk, i = i0 + di;
        const bool ok = k >= 0 && k < NZ && i >= 0 && i < NX;
        float d = 0.0f;
#pragma unroll
        for (int m = 1; m <= R; m++) {
            d = fmaf(cc[m - 1], sVX[RX::at(dk, di + m - 1)] - sVX[RX::at(dk, di - m)], d);
            d = fmaf(cc[m - 1], sVZ[RZ::at(dk + m - 1, di)] - sVZ[RZ::at(dk - m, di)], d);
        }
        float A, B;
        damp(pf.xi(di) + pf.zi(dk), A, B);
        float cp = sK[RK::at(dk, di)];
        cp *= B;
        float val = fmaf(-cp, d, A * sP[RIN::at(dk, di)]);
        if (a.hsrc && ok) {
            const float w = row_weight(k, a.src.kp, a.src.wp0, a.src.wp1);
            const int js = i - a.src.i0;
            if (w != 0.0f && js >= 0 && js < a.src.n)
                val = fmaf(cp * (w * a.src.scale), (float)__ldcg(a.hsrc + (size_t)n * a.src.n + js), val);
        }
        if (ok && in_tile(dk, di, TX, TZ)) {
            if (LAST) st_out(io.p_out + k * pitch + i, val);
            if (a.outp) {
                const float w = row_weight(k, a.rec.kp, a.rec.wp0, a.rec.wp1);
                const int jr = i - a.rec.i0;
                if (w != 0.0f && jr >= 0 && jr < a.rec.n)
                    atomicAdd(&a.outp[(size_t)n * a.rec.n + jr], (double)w * (double)val);
            }
        }
        if (!LAST) sPO[RP::at(dk, di)] = ok ? val : 0.0f;
    });
}

}  // namespace
}  // namespace ssx

namespace ssx {
namespace {

// One transposed step n over regions (reverse time): q = C_p pbar on RIN
// (into sQ; C_p in the layout RC), vbar' on RX / RZ (C_v vbar' into sCVX /
// sCVZ and, unless LAST, the new vbar = A_v vbar' into sVXO / sVZO), then
// pbar on RP. The read-outs of the transposed injection (hbar, fbar) come
// from the tile's own points; the adjoint data of step n-1 are injected at
// every point computed.
template <int TX, int TZ, int NT, class RX, class RZ, class RP, class RIN, class RXI, class RZI,
          class RC, bool LAST>
__device__ __forceinline__ void adj_regions(const AdjArgs &a, const StepIO &io, int n, int i0, int k0,
                                            const Prof<TX, TZ> &pf, const float *sP, const float *sC, float *sQ,
                                            const float *sVXI, const float *sVZI, float *sCVX,
                                            float *sCVZ, float *sVXO, float *sVZO, float *sPO) {
    constexpr int R = kR2;
    const GridArgs &g = a.g;
    const int pitch = g.pitch, NX = g.NX, NZ = g.NZ;
    float cc[R];
#pragma unroll
    for (int m = 0; m < R; m++) cc[m] = g.c[m];
    const float cv = g.cv;
    RIN::template each<NT>([&](int dk, int di) {
        sQ[RIN::at(dk, di)] = __fmul_rn(sC[RC::at(dk, di)], sP[RIN::at(dk, di)]);
    });
    __syncthreads();
    // transposed pressure injection: hbar[n] = scale sum_k w_k q (the tile's points)
    if (a.hbar) {
        Reg<0, TZ, 0, TX>::template each<NT>([&](int dk, int di) {
            const int k = k0 + dk, i = i0 + di;
            const float w = row_weight(k, a.src.kp, a.src.wp0, a.src.wp1);
            const int jl = i - a.src.i0;
            if (i < NX && w != 0.0f && jl >= 0 && jl < a.src.n)
                atomicAdd(&a.hbar[(size_t)n * a.src.n + jl],
                          (double)(w * a.src.scale) * (double)sQ[RIN::at(dk, di)]);
        });
    }
    // vbar_x' = vbar_x + D+ q
    RX::template each<NT>([&](int dk, int di) {
        const int k = k0 + dk, j = i0 + di;
        const bool ok = k >= 0 && k < NZ && j >= 0 && j < NX - 1;
        float d = 0.0f;
#pragma unroll
        for (int m = 1; m <= R; m++) d = fmaf(cc[m - 1], sQ[RIN::at(dk, di + m)] - sQ[RIN::at(dk, di + 1 - m)], d);
        const float vbx = sVXI[RXI::at(dk, di)] + d;
        float A, B;
        damp(pf.xh(di) + pf.zi(dk), A, B);
        sCVX[RX::at(dk, di)] = ok ? (B * cv) * vbx : 0.0f;
        const float ox = A * vbx;
        if (LAST) {
            if (ok && in_tile(dk, di, TX, TZ)) st_out(io.vx_out + k * pitch + j, ox);
        } else {
            sVXO[RX::at(dk, di)] = ok ? ox : 0.0f;
        }
    });
    // vbar_z' likewise; the transposed velocity injection read out, then the
    // transposed v_z sampling of step n-1 injected
    RZ::template each<NT>([&](int dk, int di) {
        const int kk = k0 + dk, i = i0 + di;
        const bool ok = i >= 0 && i < NX && kk >= 0 && kk < NZ - 1;
        float d = 0.0f;
#pragma unroll
        for (int m = 1; m <= R; m++) d = fmaf(cc[m - 1], sQ[RIN::at(dk + m, di)] - sQ[RIN::at(dk + 1 - m, di)], d);
        const float vb = sVZI[RZI::at(dk, di)] + d;
        float A, B;
        damp(pf.xi(di) + pf.zh(dk), A, B);
        const float vz = (B * cv) * vb;
        float out = A * vb;
        if (a.fbar && ok && in_tile(dk, di, TX, TZ)) {
            const float wf = row_weight(kk, a.src.kv, a.src.wv0, a.src.wv1);
            const int js = i - a.src.i0;
            if (wf != 0.0f && js >= 0 && js < a.src.n)
                atomicAdd(&a.fbar[(size_t)n * a.src.n + js], (double)(wf * a.src.scale) * (double)vz);
        }
        if (a.yv && n >= 1 && ok) {
            const float wy = row_weight(kk, a.rec.kv, a.rec.wv0, a.rec.wv1);
            const int jr = i - a.rec.i0;
            if (wy != 0.0f && jr >= 0 && jr < a.rec.n)
                out = fmaf(wy, (float)__ldcg(a.yv + (size_t)(n - 1) * a.rec.n + jr), out);
        }
        sCVZ[RZ::at(dk, di)] = ok ? vz : 0.0f;
        if (LAST) {
            if (ok && in_tile(dk, di, TX, TZ)) st_out(io.vz_out + kk * pitch + i, out);
        } else {
            sVZO[RZ::at(dk, di)] = ok ? out : 0.0f;
        }
    });
    __syncthreads();
    // pbar <- A_p pbar + D- (C_v vbar'), then the transposed p sampling of step n-1
    RP::template each<NT>([&](int dk, int di) {
        const int k = k0 + dk, i = i0 + di;
        const bool ok = k >= 0 && k < NZ && i >= 0 && i < NX;
        float d = 0.0f;
#pragma unroll
        for (int m = 1; m <= R; m++) {
            d = fmaf(cc[m - 1], sCVX[RX::at(dk, di + m - 1)] - sCVX[RX::at(dk, di - m)], d);
            d = fmaf(cc[m - 1], sCVZ[RZ::at(dk + m - 1, di)] - sCVZ[RZ::at(dk - m, di)], d);
        }
        float A, B;
        damp(pf.xi(di) + pf.zi(dk), A, B);
        float out = fmaf(A, sP[RIN::at(dk, di)], d);
        if (a.yp && n >= 1 && ok) {
            const float w = row_weight(k, a.rec.kp, a.rec.wp0, a.rec.wp1);
            const int jr = i - a.rec.i0;
            if (w != 0.0f && jr >= 0 && jr < a.rec.n)
                out = fmaf(w, (float)__ldcg(a.yp + (size_t)(n - 1) * a.rec.n + jr), out);
        }
        if (LAST) {
            if (ok && in_tile(dk, di, TX, TZ)) st_out(io.p_out + k * pitch + i, out);
        } else {
            sPO[RP::at(dk, di)] = ok ? out : 0.0f;
        }
    });
}

}  // namespace
}  // namespace ssx

namespace ssx {
namespace {

// Shared memory of a two-step launch (the transposed step uses every array,
// the forward step all but q, cvx, cvz as its own).
template <int TX, int TZ>
struct TwoSmem {
    using G = TwoRegs<TX, TZ>;
    float p0[G::P0::N];     // p^n over P0 (forward), pbar (transposed)
    float c[G::P0::N];      // kappa over P1 (forward, layout P1) or C_p over P0 (transposed)
    float q[G::P0::N];      // q = C_p pbar of the current step
    float vx0[G::VX0::N], vz0[G::VZ0::N];   // v of step A's input
    float cvx[G::VX0::N], cvz[G::VZ0::N];   // C_v vbar' (transposed); step B's v (forward)
    float vx1[G::VX0::N], vz1[G::VZ0::N];   // v after step A: step B's input
    float p1[G::P1::N];     // p after step A: step B's input
    Prof<TX, TZ> pf;        // sponge profiles
};

template <int TX, int TZ>
constexpr size_t two_smem_bytes() { return sizeof(TwoSmem<TX, TZ>); }

// Launch t of a single-sweep phase: steps 2t and 2t + 1 of the sweep (one
// step, 2t, when TWO is false: the last launch of an odd step count). Reads
// buffer t mod 2, writes the other one.
template <int TX, int TZ, int NT, bool TWO>
__global__ void __launch_bounds__(NT) k_two(const JobSet P, int t) {
    using G = TwoRegs<TX, TZ>;
    griddep_launch();
    extern __shared__ __align__(16) unsigned char ssx_two_smem[];
    TwoSmem<TX, TZ> &sm = *reinterpret_cast<TwoSmem<TX, TZ> *>(ssx_two_smem);
    const Job &J = P.job[0];
    int i0, k0;
    tile_corner<TX, TZ>(J.tx_mul, J.tx_shift, J.tiles_x, blockIdx.x, i0, k0);
    const int b = t & 1, st = 2 * t;
    StepIO io;
    io.p_in = J.f[b][0];
    io.vx_in = J.f[b][1];
    io.vz_in = J.f[b][2];
    io.p_out = J.f[b ^ 1][0];
    io.vx_out = J.f[b ^ 1][1];
    io.vz_out = J.f[b ^ 1][2];
    io.n = 0;
    if (J.adj) {
        const AdjArgs &a = J.aa;
        const GridArgs &g = a.g;
        const int pitch = g.pitch, NX = g.NX, NZ = g.NZ;
        const int n0 = J.nt - 1 - st;
        // C_p and the profiles never change during the sweep: read before the
        // grid dependency wait
        sm.pf.template load<NT>(g, i0, k0);
        if (TWO) load_region<typename G::P0, typename G::P0, NT>(sm.c, g.cpk, pitch, i0, k0, NX, NZ, true);
        else load_region<typename G::P1, typename G::P0, NT>(sm.c, g.cpk, pitch, i0, k0, NX, NZ, true);
        griddep_wait();   // the previous launch's fields are complete
        if (TWO) {
            load_region<typename G::P0, typename G::P0, NT>(sm.p0, io.p_in, pitch, i0, k0, NX, NZ, false);
            load_region<typename G::VX0, typename G::VX0, NT>(sm.vx0, io.vx_in, pitch, i0, k0, NX - 1, NZ, false);
            load_region<typename G::VZ0, typename G::VZ0, NT>(sm.vz0, io.vz_in, pitch, i0, k0, NX, NZ - 1, false);
        } else {
            load_region<typename G::P1, typename G::P1, NT>(sm.p1, io.p_in, pitch, i0, k0, NX, NZ, false);
            load_region<typename G::VXB, typename G::VX0, NT>(sm.vx1, io.vx_in, pitch, i0, k0, NX - 1, NZ, false);
            load_region<typename G::VZB, typename G::VZ0, NT>(sm.vz1, io.vz_in, pitch, i0, k0, NX, NZ - 1, false);
        }
        __syncthreads();
        if (TWO) {
            adj_regions<TX, TZ, NT, typename G::VX0, typename G::VZ0, typename G::P1, typename G::P0,
                        typename G::VX0, typename G::VZ0, typename G::P0, false>(
                a, io, n0, i0, k0, sm.pf, sm.p0, sm.c, sm.q, sm.vx0, sm.vz0, sm.cvx, sm.cvz, sm.vx1, sm.vz1, sm.p1);
            __syncthreads();
        }
        adj_regions<TX, TZ, NT, typename G::VXB, typename G::VZB, typename G::T, typename G::P1,
                    typename G::VX0, typename G::VZ0, typename G::P0, true>(
            a, io, TWO ? n0 - 1 : n0, i0, k0, sm.pf, sm.p1, sm.c, sm.q, sm.vx1, sm.vz1, sm.cvx, sm.cvz, nullptr,
            nullptr, nullptr);
    } else {
        const FwdArgs &a = J.fa;
        const GridArgs &g = a.g;
        const int pitch = g.pitch, NX = g.NX, NZ = g.NZ;
        sm.pf.template load<NT>(g, i0, k0);
        load_region<typename G::P1, typename G::P1, NT>(sm.c, g.kap, pitch, i0, k0, NX, NZ, true);
        griddep_wait();
        if (TWO) {
            load_region<typename G::P0, typename G::P0, NT>(sm.p0, io.p_in, pitch, i0, k0, NX, NZ, false);
            load_region<typename G::VX0, typename G::VX0, NT>(sm.vx0, io.vx_in, pitch, i0, k0, NX - 1, NZ, false);
            load_region<typename G::VZ0, typename G::VZ0, NT>(sm.vz0, io.vz_in, pitch, i0, k0, NX, NZ - 1, false);
        } else {
            load_region<typename G::P1, typename G::P1, NT>(sm.p1, io.p_in, pitch, i0, k0, NX, NZ, false);
            load_region<typename G::VXB, typename G::VX0, NT>(sm.vx1, io.vx_in, pitch, i0, k0, NX - 1, NZ, false);
            load_region<typename G::VZB, typename G::VZ0, NT>(sm.vz1, io.vz_in, pitch, i0, k0, NX, NZ - 1, false);
        }
        __syncthreads();
        if (TWO) {
            fwd_regions<TX, TZ, NT, typename G::VX0, typename G::VZ0, typename G::P1, typename G::P0,
                        typename G::VX0, typename G::VZ0, typename G::P1, false>(
                a, io, st, i0, k0, sm.pf, sm.p0, sm.vx0, sm.vz0, sm.c, sm.vx1, sm.vz1, sm.p1);
            __syncthreads();
        }
        fwd_regions<TX, TZ, NT, typename G::VXB, typename G::VZB, typename G::T, typename G::P1,
                    typename G::VX0, typename G::VZ0, typename G::P1, true>(
            a, io, TWO ? st + 1 : st, i0, k0, sm.pf, sm.p1, sm.vx1, sm.vz1, sm.c, sm.cvx, sm.cvz, nullptr);
    }
}

template <int TX, int TZ, int NT>
struct TwoKernel {
    static cudaError_t prepare() {
        const int b = (int)two_smem_bytes<TX, TZ>();
        cudaError_t e = cudaFuncSetAttribute(k_two<TX, TZ, NT, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, b);
        if (e != cudaSuccess) return e;
        return cudaFuncSetAttribute(k_two<TX, TZ, NT, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, b);
    }
    static cudaError_t launch(const JobSet &jobs, int total, int t, bool two, cudaStream_t s, bool pdl) {
        cudaLaunchConfig_t cfg = {};
        cfg.gridDim = dim3(total);
        cfg.blockDim = dim3(NT);
        cfg.dynamicSmemBytes = two_smem_bytes<TX, TZ>();
        cfg.stream = s;
        cudaLaunchAttribute at[1];
        at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
        at[0].val.programmaticStreamSerializationAllowed = 1;
        cfg.attrs = pdl ? at : nullptr;
        cfg.numAttrs = pdl ? 1 : 0;
        if (two) return cudaLaunchKernelEx(&cfg, k_two<TX, TZ, NT, true>, jobs, t);
        return cudaLaunchKernelEx(&cfg, k_two<TX, TZ, NT, false>, jobs, t);
    }
};

}  // namespace

const TileCfg kTwoCfgs[kNumTwoCfgs] = {
#define SSX_TWO_ROW(id, TX, TZ, NT) {TX, TZ, NT, 0},
    SSX_TWO_CONFIGS(SSX_TWO_ROW)
#undef SSX_TWO_ROW
};

cudaError_t prepare_two_kernels() {
    cudaError_t e = cudaSuccess;
#define SSX_CASE_TWO_PREP(id, TX, TZ, NT) if (e == cudaSuccess) e = TwoKernel<TX, TZ, NT>::prepare();
    SSX_TWO_CONFIGS(SSX_CASE_TWO_PREP)
#undef SSX_CASE_TWO_PREP
    return e;
}

cudaError_t launch_two(const JobSet &jobs, int total_tiles, int t, bool two, int m, cudaStream_t s,
                       bool pdl) {
    if (jobs.njobs != 1) return cudaErrorInvalidValue;
    switch (m) {
#define SSX_CASE_TWO_LAUNCH(id, TX, TZ, NT) \
    case id: return TwoKernel<TX, TZ, NT>::launch(jobs, total_tiles, t, two, s, pdl);
        SSX_TWO_CONFIGS(SSX_CASE_TWO_LAUNCH)
#undef SSX_CASE_TWO_LAUNCH
    }
    return cudaErrorInvalidValue;
}

}  // namespace ssx
