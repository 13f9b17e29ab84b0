// stencil_impl.cuh -- the tile step of the staggered-grid leapfrog and its
// exact transpose, and the whole-sweep persistent kernels, templated on the
// half order R, the tile shape TX x TZ and the CTA size NT. Included by one
// translation unit per R (stencil_r<R>.cu), which instantiates every tile
// configuration of kTileCfgs.
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
#pragma once
#include "ssx_internal.cuh"

namespace ssx {

namespace {

// Sponge factors of a point with s = (sigma_x + sigma_z) dt/2:
// B = 1/(1+s) and A = (1-s)/(1+s) = 2B - 1. The reciprocal is the hardware's
// approximate one (rcp.approx, about one unit in the last place: far below the
// f32 rounding of the fields it scales), except that s = 0 gives exactly
// B = A = 1, so that an undamped point rounds the same whether its tile takes
// the sponge path or the interior path.
__device__ __forceinline__ void damp(float s, float &A, float &B) {
    float r;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(1.0f + s));
    B = s == 0.0f ? 1.0f : r;
    A = fmaf(2.0f, B, -1.0f);
}

// Programmatic dependent launch: let the next step's grid become resident
// while this one runs, and wait here until the previous step's grid has
// finished and its writes are visible (a no-op without the launch attribute).
__device__ __forceinline__ void griddep_launch() {
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}
__device__ __forceinline__ void griddep_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }

// corner of sweep tile tl: tile row by the sweep's reciprocal of tiles_x
template <int TX, int TZ>
__device__ __forceinline__ void tile_corner(unsigned long long mul, int shift, int tiles_x, int tl,
                                            int &i0, int &k0) {
    const int q = (int)((unsigned)(((unsigned long long)(unsigned)tl * mul) >> 32) >> shift);
    i0 = (tl - q * tiles_x) * TX;
    k0 = q * TZ;
}

__device__ __forceinline__ float row_weight(int k, int k0, float w0, float w1) {
    return (k == k0) ? w0 : ((k == k0 + 1) ? w1 : 0.0f);
}


// Field loads go through L2 only (ld.global.cg): in the persistent sweep a
// neighbour CTA rewrote these lines during the previous step, and L1 is not
// coherent across SMs.
__device__ __forceinline__ float ldf(const float *p) { return __ldcg(p); }
// Field stores, explicitly global: where a kernel reads the field pointers
// from shared memory the compiler cannot tell their space and would emit
// generic stores.
__device__ __forceinline__ void st_out(float *p, float v) {
    asm volatile("st.global.cg.f32 [%0], %1;" ::"l"(p), "f"(v) : "memory");
}

template <int R, int TX, int TZ>
struct TileSmem {
    static constexpr int H = 2 * R;
    static constexpr int PW = TX + 2 * H, PH = TZ + 2 * H;
    static constexpr int VXW = TX + 2 * R - 1, VZH = TZ + 2 * R - 1;
    static constexpr int VXP = TX + 2 * R;   // row pitch of svx: whole 16-byte quads for order 8
    float sp[PH][PW];      // p^n (forward) or q = C_p pbar (transpose), tile + 2k halo
    alignas(16) float svx[TZ][VXP];    // v_x^{n+1/2} (forward) or C_vx vbar_x' (transpose)
    alignas(16) float svz[VZH][TX];    // v_z^{n+1/2} (forward) or C_vz vbar_z' (transpose)
};

// The field buffers and step index of one step (kept in registers).
struct StepIO {
    const float *p_in, *vx_in, *vz_in;
    float *p_out, *vx_out, *vz_out;
    int n;
};

// A tile is "interior" when its whole 2k-wide neighbourhood lies where every
// sponge factor is exactly 1 and every staggered point is valid: there the
// update needs neither damping factors nor bounds tests, and gives the same
// bits as the general path.
template <int R, int TX, int TZ>
__device__ __forceinline__ bool interior_tile(const GridArgs &g, int i0, int k0) {
    return i0 - 2 * R >= g.in_x0 && i0 + TX + 2 * R <= g.in_x1 && k0 - 2 * R >= g.in_z0 &&
           k0 + TZ + 2 * R <= g.in_z1;
}

// The elements of the tile + 2k halo region a thread stages (corners are
// never used and not loaded): f(slot, smem row, smem column, k - k0, i - i0)
// for each, slot a compile-time index 0 .. Staged::N - 1 once unrolled. Warp
// w takes rows w, w + NT/32, ...; lanes take columns lane, lane + 32, ...
template <int R, int TX, int TZ, int NT>
struct Staged {
    static constexpr int H = 2 * R, PW = TX + 2 * H, NW = NT / 32;
    static constexpr int NR1 = (TZ + NW - 1) / NW, NC1 = (PW + 31) / 32;      // tile rows, x halo
    static constexpr int NR2 = (2 * H + NW - 1) / NW, NC2 = (TX + 31) / 32;   // z halo rows
    static constexpr int N = NR1 * NC1 + NR2 * NC2;
    template <class F>
    __device__ __forceinline__ static void each(F &&f) {
        const int lane = threadIdx.x & 31, wy = threadIdx.x >> 5;
#pragma unroll
        for (int a = 0; a < NR1; a++)
#pragma unroll
            for (int b = 0; b < NC1; b++) {
                const int r = wy + NW * a, c = lane + 32 * b;
                if (r < TZ && c < PW) f(a * NC1 + b, r + H, c, r, c - H);
            }
#pragma unroll
        for (int a = 0; a < NR2; a++)
#pragma unroll
            for (int b = 0; b < NC2; b++) {
                const int r = wy + NW * a, c = lane + 32 * b;
                if (r < 2 * H && c < TX) {
                    const int rr = r < H ? r : r + TZ;
                    f(NR1 * NC1 + a * NC2 + b, rr, c + H, rr - H, c);
                }
            }
    }
};

// The same region by 16-byte quads, where every staged row starts on a
// 16-byte boundary (2k and the tile width multiples of 4 floats: orders 4
// and 8): f(slot, smem row, smem column, k - k0, i - i0) for each quad of 4
// consecutive columns, slot 0 .. StagedQ::N - 1 once unrolled. The quads of
// the tile rows (with their x halo) and of the z halo rows are numbered
// through the CTA's threads.
template <int R, int TX, int TZ, int NT>
struct StagedQ {
    static constexpr int H = 2 * R, PW = TX + 2 * H, Q1 = PW / 4, Q2 = TX / 4;
    static constexpr bool ok = H % 4 == 0 && TX % 4 == 0;
    static constexpr int N1 = TZ * Q1, N2 = 2 * H * Q2;
    static constexpr int NI1 = (N1 + NT - 1) / NT, NI2 = (N2 + NT - 1) / NT;
    static constexpr int N = NI1 + NI2;
    template <class F>
    __device__ __forceinline__ static void each(F &&f) {
#pragma unroll
        for (int a = 0; a < NI1; a++) {
            const int q = threadIdx.x + a * NT;
            if (N1 % NT == 0 || q < N1) {
                const int r = q / Q1, cq = q - r * Q1;
                f(a, r + H, 4 * cq, r, 4 * cq - H);
            }
        }
#pragma unroll
        for (int a = 0; a < NI2; a++) {
            const int q = threadIdx.x + a * NT;
            if (N2 % NT == 0 || q < N2) {
                const int r = q / Q2, cq = q - r * Q2;
                const int rr = r < H ? r : r + TZ;
                f(NI1 + a, rr, H + 4 * cq, rr - H, 4 * cq);
            }
        }
    }
};
__device__ __forceinline__ float4 ldf4(const float *p) { return __ldcg(reinterpret_cast<const float4 *>(p)); }

// Stage a field over tile + 2k halo; with PRE the staged value is C_p * field
// (transpose step), C_p from the grid's precomputed field (B_p kappa~ inside
// the grid, 0 outside: the storage's apron makes every address valid). The
// C_p factors may be read ahead (stage_cp, before the grid dependency wait:
// they never change during a sweep) and passed in.
template <int R, int TX, int TZ, int NT>
__device__ __forceinline__ void stage_cp(const GridArgs &g, int i0, int k0,
                                         float (&cp)[Staged<R, TX, TZ, NT>::N]) {
    const float *base = g.cpk + k0 * g.pitch + i0;
    const int pitch = g.pitch;
    Staged<R, TX, TZ, NT>::each([&](int e, int, int, int dk, int di) { cp[e] = __ldg(base + dk * pitch + di); });
}
template <int R, int TX, int TZ, int NT, bool PRE>
__device__ __forceinline__ void stage_p(const GridArgs &g, const float *f, int i0, int k0,
                                        float (&sp)[TZ + 4 * R][TX + 4 * R],
                                        const float (&cp)[Staged<R, TX, TZ, NT>::N]) {
    const float *base = f + k0 * g.pitch + i0;
    const int pitch = g.pitch;
    Staged<R, TX, TZ, NT>::each([&](int e, int sr, int sc, int dk, int di) {
        const float v = ldf(base + dk * pitch + di);
        sp[sr][sc] = PRE ? __fmul_rn(cp[e], v) : v;
    });
}
// by quads (StagedQ::ok): C_p read ahead by stage_cp4, then the field
template <int R, int TX, int TZ, int NT>
__device__ __forceinline__ void stage_cp4(const GridArgs &g, int i0, int k0,
                                          float4 (&cp)[StagedQ<R, TX, TZ, NT>::N]) {
    const float *base = g.cpk + k0 * g.pitch + i0;
    const int pitch = g.pitch;
    StagedQ<R, TX, TZ, NT>::each([&](int e, int, int, int dk, int di) {
        cp[e] = __ldg(reinterpret_cast<const float4 *>(base + dk * pitch + di));
    });
}
template <int R, int TX, int TZ, int NT, bool PRE>
__device__ __forceinline__ void stage_p4(const GridArgs &g, const float *f, int i0, int k0,
                                         float (&sp)[TZ + 4 * R][TX + 4 * R],
                                         const float4 (&cp)[StagedQ<R, TX, TZ, NT>::N]) {
    const float *base = f + k0 * g.pitch + i0;
    const int pitch = g.pitch;
    StagedQ<R, TX, TZ, NT>::each([&](int e, int sr, int sc, int dk, int di) {
        float4 v = ldf4(base + dk * pitch + di);
        if (PRE) {
            v.x = __fmul_rn(cp[e].x, v.x);
            v.y = __fmul_rn(cp[e].y, v.y);
            v.z = __fmul_rn(cp[e].z, v.z);
            v.w = __fmul_rn(cp[e].w, v.w);
        }
        *reinterpret_cast<float4 *>(&sp[sr][sc]) = v;
    });
}
template <int R, int TX, int TZ, int NT, bool SP, bool PRE>
__device__ __forceinline__ void stage_p(const GridArgs &g, const float *f, int i0, int k0,
                                        float (&sp)[TZ + 4 * R][TX + 4 * R]) {
    const float *base = f + k0 * g.pitch + i0, *cbase = g.cpk + k0 * g.pitch + i0;
    const int pitch = g.pitch;
    Staged<R, TX, TZ, NT>::each([&](int, int sr, int sc, int dk, int di) {
        const int o = dk * pitch + di;
        const float v = ldf(base + o);
        sp[sr][sc] = PRE ? __fmul_rn(__ldg(cbase + o), v) : v;
    });
}

// Per-thread point sets of a tile (compile-time counts): warp w owns rows
// w, w+8, ..; lane l owns columns l, l+32, ...
template <int R, int TX, int TZ, int NT>
struct TileShape {
    static constexpr int kWarps = NT / 32;
    static constexpr int VXW = TX + 2 * R - 1, VZH = TZ + 2 * R - 1;
    static constexpr int NRT = (TZ + kWarps - 1) / kWarps;    // tile rows per thread
    static constexpr int NRV = (VZH + kWarps - 1) / kWarps;   // v_z rows per thread
    static constexpr int NCT = (TX + 31) / 32;                // tile columns per thread
    static constexpr int NCX = (VXW + 31) / 32;               // v_x columns per thread
};

// One forward step on the TX x TZ tile at (i0, k0). Every global operand of
// the step is loaded in one batch at the start (p into shared memory, v and
// kappa into registers) so the step pays one memory latency, not one per loop
// iteration.
template <int R, int TX, int TZ, int NT, bool SP>
__device__ __forceinline__ void fwd_tile_impl(const FwdArgs &a, const StepIO &io, int i0, int k0,
                                              TileSmem<R, TX, TZ> &sm) {
    using S = TileSmem<R, TX, TZ>;
    using T = TileShape<R, TX, TZ, NT>;
    constexpr int kWarps = NT / 32;
    constexpr int H = S::H, VXW = S::VXW, VZH = S::VZH;
    griddep_wait();   // the previous step's fields are complete
    const GridArgs &g = a.g;
    const int pitch = g.pitch;
    const int lane = threadIdx.x & 31, wy = threadIdx.x >> 5;
    const int n = io.n;
    // grid scalars in registers: they are read in every element of every loop
    float cc[R];
#pragma unroll
    for (int m = 0; m < R; m++) cc[m] = g.c[m];
    const float cv = g.cv;
    const int NX = g.NX, NZ = g.NZ;

    float rvx[T::NRT][T::NCX], rvz[T::NRV][T::NCT], rk[T::NRT][T::NCT];
#pragma unroll
    for (int a_ = 0; a_ < T::NRT; a_++)
#pragma unroll
        for (int b = 0; b < T::NCX; b++) {
            const int r = wy + kWarps * a_, jj = lane + 32 * b;
            const int k = k0 + r, j = i0 - R + jj;
            const bool ok = r < TZ && jj < VXW && (!SP || (k < NZ && j >= 0 && j < NX - 1));
            rvx[a_][b] = ok ? ldf(io.vx_in + k * pitch + j) : 0.0f;
        }
#pragma unroll
    for (int a_ = 0; a_ < T::NRV; a_++)
#pragma unroll
        for (int b = 0; b < T::NCT; b++) {
            const int kk = wy + kWarps * a_, c = lane + 32 * b;
            const int k = k0 - R + kk, i = i0 + c;
            const bool ok = kk < VZH && c < TX && (!SP || (i < NX && k >= 0 && k < NZ - 1));
            rvz[a_][b] = ok ? ldf(io.vz_in + k * pitch + i) : 0.0f;
        }
#pragma unroll
    for (int a_ = 0; a_ < T::NRT; a_++)
#pragma unroll
        for (int b = 0; b < T::NCT; b++) {
            const int r = wy + kWarps * a_, c = lane + 32 * b;
            const bool ok = r < TZ && c < TX && (!SP || (k0 + r < NZ && i0 + c < NX));
            rk[a_][b] = ok ? __ldg(g.kap + (k0 + r) * pitch + i0 + c) : 0.0f;
        }
    stage_p<R, TX, TZ, NT, SP, false>(g, io.p_in, i0, k0, sm.sp);
    __syncthreads();

    // v_x^{n+1/2} on the tile rows, columns i0-k .. i0+TX+k-2
#pragma unroll
    for (int a_ = 0; a_ < T::NRT; a_++)
#pragma unroll
        for (int b = 0; b < T::NCX; b++) {
            const int r = wy + kWarps * a_, jj = lane + 32 * b;
            if (r >= TZ || jj >= VXW) continue;
            const int k = k0 + r, j = i0 - R + jj;
            float val = 0.0f;
            if (!SP || (k < NZ && j >= 0 && j < NX - 1)) {
                const float *row = &sm.sp[r + H][jj + R];
                float d = 0.0f;
#pragma unroll
                for (int m = 1; m <= R; m++) d = fmaf(cc[m - 1], row[m] - row[1 - m], d);
                if (SP) {
                    float A, B;
                    damp(__ldg(g.sxh + j) + __ldg(g.szi + k), A, B);
                    val = fmaf(-(B * cv), d, A * rvx[a_][b]);
                } else {
                    val = fmaf(-cv, d, rvx[a_][b]);
                }
                if (jj >= R && jj < R + TX) io.vx_out[k * pitch + j] = val;
            }
            sm.svx[r][jj] = val;
        }
    // v_z^{n+1/2} on rows k0-k .. k0+TZ+k-2, the tile columns
#pragma unroll
    for (int a_ = 0; a_ < T::NRV; a_++)
#pragma unroll
        for (int b = 0; b < T::NCT; b++) {
            const int kk = wy + kWarps * a_, c = lane + 32 * b;
            if (kk >= VZH || c >= TX) continue;
            const int k = k0 - R + kk, i = i0 + c;
            float val = 0.0f;
            if (!SP || (i < NX && k >= 0 && k < NZ - 1)) {
                float d = 0.0f;
#pragma unroll
                for (int m = 1; m <= R; m++)
                    d = fmaf(cc[m - 1], sm.sp[kk + R + m][c + H] - sm.sp[kk + R + 1 - m][c + H], d);
                if (SP) {
                    float A, B;
                    damp(__ldg(g.sxi + i) + __ldg(g.szh + k), A, B);
                    val = fmaf(-(B * cv), d, A * rvz[a_][b]);
                } else {
                    val = fmaf(-cv, d, rvz[a_][b]);
                }
                if (kk >= R && kk < R + TZ) io.vz_out[k * pitch + i] = val;
            }
            sm.svz[kk][c] = val;
        }
    // line rows only: vertical load f e_z delta(z - z_s), then the P v_z trace
    if (a.fsrc || a.outv) {
#pragma unroll
        for (int a_ = 0; a_ < T::NRV; a_++) {
            const int kk = wy + kWarps * a_;
            if (kk >= VZH) continue;
            const int k = k0 - R + kk;
            const bool own = (kk >= R && kk < R + TZ);
            const float wi = a.fsrc ? row_weight(k, a.src.kv, a.src.wv0, a.src.wv1) : 0.0f;
            const float ws = (a.outv && own) ? row_weight(k, a.rec.kv, a.rec.wv0, a.rec.wv1) : 0.0f;
            if (wi == 0.0f && ws == 0.0f) continue;
#pragma unroll
            for (int b = 0; b < T::NCT; b++) {
                const int c = lane + 32 * b;
                if (c >= TX) continue;
                const int i = i0 + c;
                if (SP && !(i < NX && k >= 0 && k < NZ - 1)) continue;
                float val = sm.svz[kk][c];
                const int js = i - a.src.i0;
                if (wi != 0.0f && js >= 0 && js < a.src.n) {
                    float cvz = cv;
                    if (SP) {
                        float A, B;
                        damp(__ldg(g.sxi + i) + __ldg(g.szh + k), A, B);
                        cvz = B * cv;
                    }
                    val = fmaf(cvz * (wi * a.src.scale), (float)a.fsrc[(size_t)n * a.src.n + js], val);
                    sm.svz[kk][c] = val;
                    if (own) io.vz_out[k * pitch + i] = val;
                }
                const int jr = i - a.rec.i0;
                if (ws != 0.0f && jr >= 0 && jr < a.rec.n)
                    atomicAdd(&a.outv[(size_t)n * a.rec.n + jr], (double)ws * (double)val);
            }
        }
    }
    __syncthreads();

    // p^{n+1} on the tile
    float pv[T::NRT][T::NCT], cpv[T::NRT][T::NCT];
#pragma unroll
    for (int a_ = 0; a_ < T::NRT; a_++)
#pragma unroll
        for (int b = 0; b < T::NCT; b++) {
            pv[a_][b] = 0.0f;
            cpv[a_][b] = 0.0f;
            const int r = wy + kWarps * a_, c = lane + 32 * b;
            if (r >= TZ || c >= TX) continue;
            const int k = k0 + r, i = i0 + c;
            if (!SP || (k < NZ && i < NX)) {
                float d = 0.0f;
#pragma unroll
                for (int m = 1; m <= R; m++) {
                    d = fmaf(cc[m - 1], sm.svx[r][c + R + m - 1] - sm.svx[r][c + R - m], d);
                    d = fmaf(cc[m - 1], sm.svz[r + R + m - 1][c] - sm.svz[r + R - m][c], d);
                }
                float cp = rk[a_][b], A = 1.0f;
                if (SP) {
                    float B;
                    damp(__ldg(g.sxi + i) + __ldg(g.szi + k), A, B);
                    cp *= B;
                }
                const float val = fmaf(-cp, d, SP ? A * sm.sp[r + H][c + H] : sm.sp[r + H][c + H]);
                io.p_out[k * pitch + i] = val;
                pv[a_][b] = val;
                cpv[a_][b] = cp;
            }
        }
    // line rows only: constitutive defect h delta(z - z_s), then the P p trace
    if (a.hsrc || a.outp) {
#pragma unroll
        for (int a_ = 0; a_ < T::NRT; a_++) {
            const int r = wy + kWarps * a_;
            if (r >= TZ) continue;
            const int k = k0 + r;
            const float wi = a.hsrc ? row_weight(k, a.src.kp, a.src.wp0, a.src.wp1) : 0.0f;
            const float ws = a.outp ? row_weight(k, a.rec.kp, a.rec.wp0, a.rec.wp1) : 0.0f;
            if (wi == 0.0f && ws == 0.0f) continue;
#pragma unroll
            for (int b = 0; b < T::NCT; b++) {
                const int c = lane + 32 * b;
                if (c >= TX) continue;
                const int i = i0 + c;
                if (SP && !(k < NZ && i < NX)) continue;
                float val = pv[a_][b];
                const int js = i - a.src.i0;
                if (wi != 0.0f && js >= 0 && js < a.src.n) {
                    val = fmaf(cpv[a_][b] * (wi * a.src.scale), (float)a.hsrc[(size_t)n * a.src.n + js], val);
                    io.p_out[k * pitch + i] = val;
                }
                const int jr = i - a.rec.i0;
                if (ws != 0.0f && jr >= 0 && jr < a.rec.n)
                    atomicAdd(&a.outp[(size_t)n * a.rec.n + jr], (double)ws * (double)val);
            }
        }
    }
}

// One transposed step on the tile at (i0, k0) (same batching of loads).
template <int R, int TX, int TZ, int NT, bool SP>
__device__ __forceinline__ void adj_tile_impl(const AdjArgs &a, const StepIO &io, int i0, int k0,
                                              TileSmem<R, TX, TZ> &sm) {
    using S = TileSmem<R, TX, TZ>;
    using T = TileShape<R, TX, TZ, NT>;
    constexpr int kWarps = NT / 32;
    constexpr int H = S::H, VXW = S::VXW, VZH = S::VZH;
    griddep_wait();   // the previous step's fields are complete
    const GridArgs &g = a.g;
    const int pitch = g.pitch;
    const int lane = threadIdx.x & 31, wy = threadIdx.x >> 5;
    const int n = io.n;
    // grid scalars in registers: they are read in every element of every loop
    float cc[R];
#pragma unroll
    for (int m = 0; m < R; m++) cc[m] = g.c[m];
    const float cv = g.cv;
    const int NX = g.NX, NZ = g.NZ;

    float rvx[T::NRT][T::NCX], rvz[T::NRV][T::NCT], rp[T::NRT][T::NCT];
#pragma unroll
    for (int a_ = 0; a_ < T::NRT; a_++)
#pragma unroll
        for (int b = 0; b < T::NCX; b++) {
            const int r = wy + kWarps * a_, jj = lane + 32 * b;
            const int k = k0 + r, j = i0 - R + jj;
            const bool ok = r < TZ && jj < VXW && (!SP || (k < NZ && j >= 0 && j < NX - 1));
            rvx[a_][b] = ok ? ldf(io.vx_in + k * pitch + j) : 0.0f;
        }
#pragma unroll
    for (int a_ = 0; a_ < T::NRV; a_++)
#pragma unroll
        for (int b = 0; b < T::NCT; b++) {
            const int kk = wy + kWarps * a_, c = lane + 32 * b;
            const int k = k0 - R + kk, i = i0 + c;
            const bool ok = kk < VZH && c < TX && (!SP || (i < NX && k >= 0 && k < NZ - 1));
            rvz[a_][b] = ok ? ldf(io.vz_in + k * pitch + i) : 0.0f;
        }
#pragma unroll
    for (int a_ = 0; a_ < T::NRT; a_++)
#pragma unroll
        for (int b = 0; b < T::NCT; b++) {
            const int r = wy + kWarps * a_, c = lane + 32 * b;
            const bool ok = r < TZ && c < TX && (!SP || (k0 + r < NZ && i0 + c < NX));
            rp[a_][b] = ok ? ldf(io.p_in + (k0 + r) * pitch + i0 + c) : 0.0f;
        }
    // q = C_p pbar over tile + 2k halo
    stage_p<R, TX, TZ, NT, SP, true>(g, io.p_in, i0, k0, sm.sp);
    __syncthreads();
    // transposed pressure injection: hbar[n] = scale * sum_k w_k q (tile only)
    if (a.hbar) {
#pragma unroll
        for (int a_ = 0; a_ < T::NRT; a_++) {
            const int r = wy + kWarps * a_;
            const int k = k0 + r;
            const float w = r < TZ ? row_weight(k, a.src.kp, a.src.wp0, a.src.wp1) : 0.0f;
            if (w != 0.0f) {
#pragma unroll
                for (int b = 0; b < T::NCT; b++) {
                    const int c = lane + 32 * b;
                    const int i = i0 + c, jl = i - a.src.i0;
                    if (c < TX && i < NX && jl >= 0 && jl < a.src.n)
                        atomicAdd(&a.hbar[(size_t)n * a.src.n + jl],
                                  (double)(w * a.src.scale) * (double)sm.sp[r + H][c + H]);
                }
            }
        }
    }

    // vbar_x' = vbar_x + D+ q; keep C_vx vbar_x' for the p update
#pragma unroll
    for (int a_ = 0; a_ < T::NRT; a_++)
#pragma unroll
        for (int b = 0; b < T::NCX; b++) {
            const int r = wy + kWarps * a_, jj = lane + 32 * b;
            if (r >= TZ || jj >= VXW) continue;
            const int k = k0 + r, j = i0 - R + jj;
            float val = 0.0f;
            if (!SP || (k < NZ && j >= 0 && j < NX - 1)) {
                const float *row = &sm.sp[r + H][jj + R];
                float d = 0.0f;
#pragma unroll
                for (int m = 1; m <= R; m++) d = fmaf(cc[m - 1], row[m] - row[1 - m], d);
                const float vb = rvx[a_][b] + d;
                if (SP) {
                    float A, B;
                    damp(__ldg(g.sxh + j) + __ldg(g.szi + k), A, B);
                    val = (B * cv) * vb;
                    if (jj >= R && jj < R + TX) io.vx_out[k * pitch + j] = A * vb;
                } else {
                    val = cv * vb;
                    if (jj >= R && jj < R + TX) io.vx_out[k * pitch + j] = vb;
                }
            }
            sm.svx[r][jj] = val;
        }
    // vbar_z' likewise
    float ov[T::NRV][T::NCT];
#pragma unroll
    for (int a_ = 0; a_ < T::NRV; a_++)
#pragma unroll
        for (int b = 0; b < T::NCT; b++) {
            ov[a_][b] = 0.0f;
            const int kk = wy + kWarps * a_, c = lane + 32 * b;
            if (kk >= VZH || c >= TX) continue;
            const int k = k0 - R + kk, i = i0 + c;
            float val = 0.0f;
            if (!SP || (i < NX && k >= 0 && k < NZ - 1)) {
                float d = 0.0f;
#pragma unroll
                for (int m = 1; m <= R; m++)
                    d = fmaf(cc[m - 1], sm.sp[kk + R + m][c + H] - sm.sp[kk + R + 1 - m][c + H], d);
                const float vb = rvz[a_][b] + d;
                float A = 1.0f, B = 1.0f;
                if (SP) damp(__ldg(g.sxi + i) + __ldg(g.szh + k), A, B);
                val = (B * cv) * vb;
                if (kk >= R && kk < R + TZ) {
                    const float out = SP ? A * vb : vb;
                    io.vz_out[k * pitch + i] = out;
                    ov[a_][b] = out;
                }
            }
            sm.svz[kk][c] = val;
        }
    // line rows only: the transposed velocity injection read out, and the
    // transposed sampling of step n-1 added to the outgoing state
    if (a.fbar || (a.yv && n >= 1)) {
#pragma unroll
        for (int a_ = 0; a_ < T::NRV; a_++) {
            const int kk = wy + kWarps * a_;
            if (kk >= VZH || kk < R || kk >= R + TZ) continue;
            const int k = k0 - R + kk;
            const float wf = a.fbar ? row_weight(k, a.src.kv, a.src.wv0, a.src.wv1) : 0.0f;
            const float wy_ = (a.yv && n >= 1) ? row_weight(k, a.rec.kv, a.rec.wv0, a.rec.wv1) : 0.0f;
            if (wf == 0.0f && wy_ == 0.0f) continue;
#pragma unroll
            for (int b = 0; b < T::NCT; b++) {
                const int c = lane + 32 * b;
                if (c >= TX) continue;
                const int i = i0 + c;
                if (SP && !(i < NX && k >= 0 && k < NZ - 1)) continue;
                const int js = i - a.src.i0;
                if (wf != 0.0f && js >= 0 && js < a.src.n)
                    atomicAdd(&a.fbar[(size_t)n * a.src.n + js],
                              (double)(wf * a.src.scale) * (double)sm.svz[kk][c]);
                const int jr = i - a.rec.i0;
                if (wy_ != 0.0f && jr >= 0 && jr < a.rec.n)
                    io.vz_out[k * pitch + i] =
                        fmaf(wy_, (float)a.yv[(size_t)(n - 1) * a.rec.n + jr], ov[a_][b]);
            }
        }
    }
    __syncthreads();

    // pbar <- A_p pbar + D- (C_v vbar')
    float po[T::NRT][T::NCT];
#pragma unroll
    for (int a_ = 0; a_ < T::NRT; a_++)
#pragma unroll
        for (int b = 0; b < T::NCT; b++) {
            po[a_][b] = 0.0f;
            const int r = wy + kWarps * a_, c = lane + 32 * b;
            if (r >= TZ || c >= TX) continue;
            const int k = k0 + r, i = i0 + c;
            if (!SP || (k < NZ && i < NX)) {
                float d = 0.0f;
#pragma unroll
                for (int m = 1; m <= R; m++) {
                    d = fmaf(cc[m - 1], sm.svx[r][c + R + m - 1] - sm.svx[r][c + R - m], d);
                    d = fmaf(cc[m - 1], sm.svz[r + R + m - 1][c] - sm.svz[r + R - m][c], d);
                }
                float out;
                if (SP) {
                    float A, B;
                    damp(__ldg(g.sxi + i) + __ldg(g.szi + k), A, B);
                    out = fmaf(A, rp[a_][b], d);
                } else {
                    out = rp[a_][b] + d;
                }
                io.p_out[k * pitch + i] = out;
                po[a_][b] = out;
            }
        }
    // line rows only: the transposed pressure sampling of step n-1
    if (a.yp && n >= 1) {
#pragma unroll
        for (int a_ = 0; a_ < T::NRT; a_++) {
            const int r = wy + kWarps * a_;
            if (r >= TZ) continue;
            const int k = k0 + r;
            const float w = row_weight(k, a.rec.kp, a.rec.wp0, a.rec.wp1);
            if (w == 0.0f) continue;
#pragma unroll
            for (int b = 0; b < T::NCT; b++) {
                const int c = lane + 32 * b;
                if (c >= TX) continue;
                const int i = i0 + c;
                if (SP && !(k < NZ && i < NX)) continue;
                const int jr = i - a.rec.i0;
                if (jr >= 0 && jr < a.rec.n)
                    io.p_out[k * pitch + i] =
                        fmaf(w, (float)a.yp[(size_t)(n - 1) * a.rec.n + jr], po[a_][b]);
            }
        }
    }
}

// ---------------------------------------------------------------------------
// Tiles by column strips. Thread t owns tile column c = t % TX and the L rows
// [s L, s L + L) of strip s = t / TX. Its v_z comes from a register window of
// L + 2k - 1 values down its column (instead of 2k shared-memory reads per
// point), the z part of its pressure update from a window over the v_z rows,
// and its own old pressures from the first window; only the x differences read
// shared memory per point. The damping factors' column parts are loaded once
// per thread and the row parts once per row. The halo values of v (2k-1
// columns of v_x, 2k-1 rows of v_z) are shared out over all threads.
//
// SP: the tile meets the sponge or the grid edge (damping and masks);
// LN: a line row (injection or sampling) meets the tile. Every point's
// arithmetic is the per-point arithmetic of fwd_tile_impl / adj_tile_impl,
// term for term, so results do not depend on the tile shape.
// ---------------------------------------------------------------------------
template <int R, int TX, int TZ, int NT>
struct StripShape {
    static constexpr int NS = NT / TX;                 // strips per tile
    static constexpr int L = NS > 0 ? TZ / NS : 0;     // rows per strip
    static constexpr bool ok = (NT % TX == 0) && NS >= 1 && (TZ % NS == 0) && L >= 2;
    static constexpr int NHR = 2 * R - 1;              // halo rows of v_z, halo columns of v_x
    // v_x halo: TZ rows x NHR columns, the columns padded to a power of two
    static constexpr int HXP = NHR <= 1 ? 1 : NHR <= 2 ? 2 : NHR <= 4 ? 4 : 8;
    static constexpr int NQX = (TZ * HXP + NT - 1) / NT;   // v_x halo items per thread
    // v_z halo: strip s of column c takes halo rows s, s + NS, ...
    static constexpr int NQZ = NS > 0 ? (NHR + NS - 1) / NS : 0;
};

// rows kl, kl + 1 of a line against the rows [lo, hi)
__device__ __forceinline__ bool line_hits(int kl, int lo, int hi) { return kl + 1 >= lo && kl < hi; }

template <int R, int TZ>
__device__ __forceinline__ bool fwd_lines(const FwdArgs &a, int k0) {
    return (a.fsrc && line_hits(a.src.kv, k0 - R, k0 + TZ + R - 1)) ||
           (a.hsrc && line_hits(a.src.kp, k0, k0 + TZ)) ||
           (a.outv && line_hits(a.rec.kv, k0, k0 + TZ)) ||
           (a.outp && line_hits(a.rec.kp, k0, k0 + TZ));
}

template <int TZ>
__device__ __forceinline__ bool adj_lines(const AdjArgs &a, int k0, int n) {
    return (a.hbar && line_hits(a.src.kp, k0, k0 + TZ)) ||
           (a.fbar && line_hits(a.src.kv, k0, k0 + TZ)) ||
           (a.yv && n >= 1 && line_hits(a.rec.kv, k0, k0 + TZ)) ||
           (a.yp && n >= 1 && line_hits(a.rec.kp, k0, k0 + TZ));
}

// Strip geometry of one thread and its halo items. In a sponge tile every
// load is made (the field storage has an apron of zeros around the padded
// grid, so all addresses are inside it) and points outside the grid are
// masked afterwards, which keeps the element loops free of branches.
template <int R, int TX, int TZ, int NT>
struct StripThread {
    using Q = StripShape<R, TX, TZ, NT>;
    int c, rs, i;
    int hx_r[Q::NQX], hx_jj[Q::NQX];    // v_x halo: tile row, v_x column (-1: none)
    int hz_kk[Q::NQZ];                  // v_z halo: v_z row (-1: none)
    __device__ __forceinline__ StripThread(int i0) {
        const int t = threadIdx.x;
        c = t % TX;
        rs = (t / TX) * Q::L;
        i = i0 + c;
#pragma unroll
        for (int q = 0; q < Q::NQX; q++) {
            const int e = t + q * NT, hx = e % Q::HXP;   // power of two: mask and shift
            hx_r[q] = e / Q::HXP;
            hx_jj[q] = (hx < Q::NHR && e < TZ * Q::HXP) ? (hx < R ? hx : hx + TX) : -1;
        }
#pragma unroll
        for (int q = 0; q < Q::NQZ; q++) {
            const int hz = t / TX + q * Q::NS;
            hz_kk[q] = hz < Q::NHR ? (hz < R ? hz : hz + TZ) : -1;
        }
    }
};

// Operands of a strip step read straight from the field storage (the tile's
// p, or q = C_p pbar, is staged into shared memory by stage_p). `own_*(j)`:
// the thread's column at strip row j; `hvx(r, jj)`: v_x at tile row r and
// v_x column jj (x = i0 - k + jj); `hvz(kk)`: v_z at row k0 - k + kk of the
// thread's column.
template <int R, int TX, int TZ, int NT, bool SP>
struct GlobalIn {
    // false: the forward step's p is staged by all threads of the CTA
    static constexpr bool kStaged = false;
    const GridArgs &g;
    const StepIO &io;
    const int i0, k0, pitch;
    const float *vxp, *vzp, *kp, *pp;
    float (&spa)[TZ + 4 * R][TX + 4 * R];
    // the sweep's injected gathers were complete before the launch chain
    // began (no sweep of the phase produces them): the step may read its
    // line values before the grid dependency wait, with the constants
    const bool lines_ready;
    __device__ __forceinline__ GlobalIn(const GridArgs &g_, const StepIO &io_, int i0_, int k0_,
                                        int rs, int c, TileSmem<R, TX, TZ> &sm, bool lines_ready_)
        : g(g_), io(io_), i0(i0_), k0(k0_), pitch(g_.pitch), spa(sm.sp), lines_ready(lines_ready_) {
        const int o0 = (k0 + rs) * pitch + i0 + c;
        vxp = io.vx_in + o0;
        vzp = io.vz_in + o0;
        kp = g.kap + o0;
        pp = io.p_in + o0;
    }
    __device__ __forceinline__ float own_vx(int j) const { return ldf(vxp + j * pitch); }
    __device__ __forceinline__ float own_vz(int j) const { return ldf(vzp + j * pitch); }
    __device__ __forceinline__ float own_kap(int j) const { return __ldg(kp + j * pitch); }
    __device__ __forceinline__ float own_p(int j) const { return ldf(pp + j * pitch); }
    __device__ __forceinline__ float hvx(int r, int jj) const {
        return ldf(io.vx_in + (k0 + r) * pitch + (i0 - R + jj));
    }
    __device__ __forceinline__ float hvz(int kk, int i) const {
        return ldf(io.vz_in + (k0 - R + kk) * pitch + i);
    }
    // by quads (fwd_quad / adj_quad): v_x at tile row r from v_x column jj,
    // v_z at v_z row kk, kappa and p at tile row r, from tile column c4
    __device__ __forceinline__ float4 vx4(int r, int jj) const {
        return ldf4(io.vx_in + (k0 + r) * pitch + (i0 - R + jj));
    }
    __device__ __forceinline__ float4 vz4(int kk, int c4) const {
        return ldf4(io.vz_in + (k0 - R + kk) * pitch + i0 + c4);
    }
    __device__ __forceinline__ float4 kap4(int r, int c4) const {
        return __ldg(reinterpret_cast<const float4 *>(g.kap + (k0 + r) * pitch + i0 + c4));
    }
    __device__ __forceinline__ float4 p4(int r, int c4) const { return ldf4(io.p_in + (k0 + r) * pitch + i0 + c4); }
    // the transposed step's C_p factors of the staged region, read before the
    // grid dependency wait (set-up data, unchanged by the previous step) where
    // the register budget allows it (CTAs of up to 256 threads); larger CTAs
    // read them with the field
    static constexpr bool kCpAhead = NT <= 256;
    // the grid's constants are read ahead of the wait in CTAs of up to 256
    // threads; larger CTAs (64 registers a thread) wait first, so that the
    // constants need not stay live across the wait
    static constexpr bool kAhead = NT <= 256;
    // orders 4 and 8 stage by 16-byte quads
    static constexpr bool kQuad = StagedQ<R, TX, TZ, NT>::ok;
    using SQ = StagedQ<R, TX, TZ, NT>;
    float cpre[kQuad ? 1 : Staged<R, TX, TZ, NT>::N];
    float4 cpre4[kQuad ? SQ::N : 1];
    template <bool PRE>
    __device__ __forceinline__ void prestage() {
        if (PRE && kCpAhead) {
            if constexpr (kQuad) stage_cp4<R, TX, TZ, NT>(g, i0, k0, cpre4);
            else stage_cp<R, TX, TZ, NT>(g, i0, k0, cpre);
        }
    }
    // the previous step's fields are complete from here on
    __device__ __forceinline__ void wait() const { griddep_wait(); }
    template <bool PRE>
    __device__ __forceinline__ void stage() {
        if constexpr (kQuad) {
            if (PRE && !kCpAhead) stage_cp4<R, TX, TZ, NT>(g, i0, k0, cpre4);
            stage_p4<R, TX, TZ, NT, PRE>(g, io.p_in, i0, k0, spa, cpre4);
        } else if (kCpAhead) {
            stage_p<R, TX, TZ, NT, PRE>(g, io.p_in, i0, k0, spa, reinterpret_cast<const float(&)[Staged<R, TX, TZ, NT>::N]>(cpre));
        } else {
            stage_p<R, TX, TZ, NT, SP, PRE>(g, io.p_in, i0, k0, spa);
        }
    }
    __device__ __forceinline__ float (&sp())[TZ + 4 * R][TX + 4 * R] { return spa; }
};

template <int R, int TX, int TZ, int NT, bool SP, bool LN, class In, class Work>
__device__ __forceinline__ void fwd_strip(const FwdArgs &a, const StepIO &io, int i0, int k0,
                                          In &in, Work &sm) {
    using S = TileSmem<R, TX, TZ>;
    using Q = StripShape<R, TX, TZ, NT>;
    constexpr int H = S::H, L = Q::L, W = L + 2 * R - 1;
    const GridArgs &g = a.g;
    const int pitch = g.pitch, NX = g.NX, NZ = g.NZ;
    const StripThread<R, TX, TZ, NT> th(i0);
    const int c = th.c, rs = th.rs, i = th.i;
    const int n = io.n;
    float cc[R];
#pragma unroll
    for (int m = 0; m < R; m++) cc[m] = g.c[m];
    const float cv = g.cv;
    const bool colp = !SP || i < NX;        // p, v_z column inside the grid
    const bool colx = !SP || i < NX - 1;    // v_x column inside the grid

    // every global operand of the step, in two batches: the grid's constants
    // (kappa, sponge profiles) before the wait for the previous step, the
    // fields after it
    float rvx[L], rvz[L], rk[L], rhx[Q::NQX], rhz[Q::NQZ];
    float sxi = 0.0f, sxh = 0.0f, szi[L], szh[L];
    if (!In::kAhead) in.wait();
    if (SP) {
        sxi = __ldg(g.sxi + min(i, NX - 1));   // clamped: masked points take any value
        sxh = __ldg(g.sxh + min(i, NX - 1));
    }
#pragma unroll
    for (int j = 0; j < L; j++) {
        const int k = k0 + rs + j;
        rk[j] = in.own_kap(j);
        if (SP) {
            szi[j] = __ldg(g.szi + min(k, NZ - 1));
            szh[j] = __ldg(g.szh + min(k, NZ - 1));
        }
    }
    // the line's values injected at this step in the thread's column (the
    // same for every row the line's weights reach): with the constants when
    // they are ready before the wait, else with the fields after it
    const int js = i - a.src.i0;
    const bool jsin = LN && js >= 0 && js < a.src.n;
    float fsv = 0.0f, hsv = 0.0f;
    auto line_values = [&]() {
        if (jsin && a.fsrc) fsv = (float)__ldcg(a.fsrc + (size_t)n * a.src.n + js);
        if (jsin && a.hsrc) hsv = (float)__ldcg(a.hsrc + (size_t)n * a.src.n + js);
    };
    if (LN && in.lines_ready) line_values();
    if (In::kAhead) in.wait();
    if (LN && !in.lines_ready) line_values();
#pragma unroll
    for (int j = 0; j < L; j++) {
        rvx[j] = in.own_vx(j);
        rvz[j] = in.own_vz(j);
    }
#pragma unroll
    for (int q = 0; q < Q::NQX; q++) rhx[q] = th.hx_jj[q] >= 0 ? in.hvx(th.hx_r[q], th.hx_jj[q]) : 0.0f;
#pragma unroll
    for (int q = 0; q < Q::NQZ; q++) rhz[q] = th.hz_kk[q] >= 0 ? in.hvz(th.hz_kk[q], i) : 0.0f;
    in.template stage<false>();
    if (!In::kStaged) __syncthreads();   // p staged by all threads
    float (&spa)[TZ + 4 * R][TX + 4 * R] = in.sp();

    // own strip: v_z from a window down the column, v_x from the row
    float pw[W];
#pragma unroll
    for (int w = 0; w < W; w++) pw[w] = spa[rs - R + 1 + w + H][c + H];
#pragma unroll
    for (int j = 0; j < L; j++) {
        const int r = rs + j, k = k0 + r;
        const bool okz = !SP || (colp && k < NZ - 1);
        float d = 0.0f;
#pragma unroll
        for (int m = 1; m <= R; m++) d = fmaf(cc[m - 1], pw[j + R - 1 + m] - pw[j + R - m], d);
        float vz, cvz = cv;
        if (SP) {
            float A, B;
            damp(sxi + szh[j], A, B);
            cvz = B * cv;
            vz = fmaf(-cvz, d, A * rvz[j]);
        } else {
            vz = fmaf(-cv, d, rvz[j]);
        }
        if (LN && a.fsrc && okz) {   // vertical load f e_z delta(z - z_s)
            const float w = row_weight(k, a.src.kv, a.src.wv0, a.src.wv1);
            if (w != 0.0f && jsin) vz = fmaf(cvz * (w * a.src.scale), fsv, vz);
        }
        if (SP) vz = okz ? vz : 0.0f;
        if (okz) st_out(io.vz_out + k * pitch + i, vz);
        if (LN && a.outv && okz) {   // P v_z trace
            const float w = row_weight(k, a.rec.kv, a.rec.wv0, a.rec.wv1);
            const int jr = i - a.rec.i0;
            if (w != 0.0f && jr >= 0 && jr < a.rec.n)
                atomicAdd(&a.outv[(size_t)n * a.rec.n + jr], (double)w * (double)vz);
        }
        sm.svz[r + R][c] = vz;

        const bool okx = !SP || (colx && k < NZ);
        const float *row = &spa[r + H][c + H];
        d = 0.0f;
#pragma unroll
        for (int m = 1; m <= R; m++) d = fmaf(cc[m - 1], row[m] - row[1 - m], d);
        float vx;
        if (SP) {
            float A, B;
            damp(sxh + szi[j], A, B);
            vx = fmaf(-(B * cv), d, A * rvx[j]);
            vx = okx ? vx : 0.0f;
        } else {
            vx = fmaf(-cv, d, rvx[j]);
        }
        if (okx) st_out(io.vx_out + k * pitch + i, vx);
        sm.svx[r][c + R] = vx;
    }
    // halo v (not written out)
#pragma unroll
    for (int q = 0; q < Q::NQX; q++) {
        const int jj = th.hx_jj[q], r = th.hx_r[q];
        if (jj < 0) continue;
        const int k = k0 + r, j = i0 - R + jj;
        const float *row = &spa[r + H][jj + R];
        float d = 0.0f;
#pragma unroll
        for (int m = 1; m <= R; m++) d = fmaf(cc[m - 1], row[m] - row[1 - m], d);
        float val;
        if (SP) {
            const bool ok = k < NZ && j >= 0 && j < NX - 1;
            float A, B;
            damp(__ldg(g.sxh + (ok ? j : 0)) + __ldg(g.szi + (ok ? k : 0)), A, B);
            val = ok ? fmaf(-(B * cv), d, A * rhx[q]) : 0.0f;
        } else {
            val = fmaf(-cv, d, rhx[q]);
        }
        sm.svx[r][jj] = val;
    }
#pragma unroll
    for (int q = 0; q < Q::NQZ; q++) {
        const int kk = th.hz_kk[q];
        if (kk < 0) continue;
        const int k = k0 - R + kk;
        float d = 0.0f;
#pragma unroll
        for (int m = 1; m <= R; m++)
            d = fmaf(cc[m - 1], spa[kk + R + m][c + H] - spa[kk + R + 1 - m][c + H], d);
        const bool ok = !SP || (colp && k >= 0 && k < NZ - 1);
        float val, cvz = cv;
        if (SP) {
            float A, B;
            damp(sxi + __ldg(g.szh + (ok ? k : 0)), A, B);
            cvz = B * cv;
            val = fmaf(-cvz, d, A * rhz[q]);
        } else {
            val = fmaf(-cv, d, rhz[q]);
        }
        if (LN && a.fsrc && ok) {
            const float w = row_weight(k, a.src.kv, a.src.wv0, a.src.wv1);
            if (w != 0.0f && jsin) val = fmaf(cvz * (w * a.src.scale), fsv, val);
        }
        sm.svz[kk][c] = ok ? val : 0.0f;
    }
    __syncthreads();

    // own strip: p^{n+1}; z differences from a window over the v_z rows
    float zw[W];
#pragma unroll
    for (int w = 0; w < W; w++) zw[w] = sm.svz[rs + w][c];
#pragma unroll
    for (int j = 0; j < L; j++) {
        const int r = rs + j, k = k0 + r;
        const bool okp = !SP || (colp && k < NZ);
        float d = 0.0f;
#pragma unroll
        for (int m = 1; m <= R; m++) {
            d = fmaf(cc[m - 1], sm.svx[r][c + R + m - 1] - sm.svx[r][c + R - m], d);
            d = fmaf(cc[m - 1], zw[j + R + m - 1] - zw[j + R - m], d);
        }
        float cp = rk[j], val;
        if (SP) {
            float A, B;
            damp(sxi + szi[j], A, B);
            cp *= B;
            val = fmaf(-cp, d, A * pw[j + R - 1]);
        } else {
            val = fmaf(-cp, d, pw[j + R - 1]);
        }
        if (LN && a.hsrc && okp) {   // constitutive defect h delta(z - z_s)
            const float w = row_weight(k, a.src.kp, a.src.wp0, a.src.wp1);
            if (w != 0.0f && jsin) val = fmaf(cp * (w * a.src.scale), hsv, val);
        }
        if (okp) st_out(io.p_out + k * pitch + i, val);
        if (LN && a.outp && okp) {   // P p trace
            const float w = row_weight(k, a.rec.kp, a.rec.wp0, a.rec.wp1);
            const int jr = i - a.rec.i0;
            if (w != 0.0f && jr >= 0 && jr < a.rec.n)
                atomicAdd(&a.outp[(size_t)n * a.rec.n + jr], (double)w * (double)val);
        }
    }
}

// The transposed step by column strips (same split of the work as fwd_strip;
// per point the arithmetic of adj_tile_impl).
template <int R, int TX, int TZ, int NT, bool SP, bool LN, class In, class Work>
__device__ __forceinline__ void adj_strip(const AdjArgs &a, const StepIO &io, int i0, int k0,
                                          In &in, Work &sm) {
    using S = TileSmem<R, TX, TZ>;
    using Q = StripShape<R, TX, TZ, NT>;
    constexpr int H = S::H, L = Q::L, W = L + 2 * R - 1;
    const GridArgs &g = a.g;
    const int pitch = g.pitch, NX = g.NX, NZ = g.NZ;
    const StripThread<R, TX, TZ, NT> th(i0);
    const int c = th.c, rs = th.rs, i = th.i;
    const int n = io.n;
    float cc[R];
#pragma unroll
    for (int m = 0; m < R; m++) cc[m] = g.c[m];
    const float cv = g.cv;
    const bool colp = !SP || i < NX;
    const bool colx = !SP || i < NX - 1;

    float rvx[L], rvz[L], rp[L], rhx[Q::NQX], rhz[Q::NQZ];
    float sxi = 0.0f, sxh = 0.0f, szi[L], szh[L];
    if (!In::kAhead) in.wait();
    if (SP) {
        sxi = __ldg(g.sxi + min(i, NX - 1));   // clamped: masked points take any value
        sxh = __ldg(g.sxh + min(i, NX - 1));
    }
#pragma unroll
    for (int j = 0; j < L; j++) {
        const int k = k0 + rs + j;
        if (SP) {
            szi[j] = __ldg(g.szi + min(k, NZ - 1));
            szh[j] = __ldg(g.szh + min(k, NZ - 1));
        }
    }
    in.template prestage<true>();   // C_p of the staged region (constants)
    // the adjoint data of step n-1 injected in the thread's column (both of
    // a line's rows take the same value): with the constants when they are
    // ready before the wait, else with the fields after it
    const int jr = i - a.rec.i0;
    const bool jrin = LN && n >= 1 && jr >= 0 && jr < a.rec.n;
    float yvv = 0.0f, ypv = 0.0f;
    auto line_values = [&]() {
        if (jrin && a.yv) yvv = (float)__ldcg(a.yv + (size_t)(n - 1) * a.rec.n + jr);
        if (jrin && a.yp) ypv = (float)__ldcg(a.yp + (size_t)(n - 1) * a.rec.n + jr);
    };
    if (LN && in.lines_ready) line_values();
    if (In::kAhead) in.wait();
    if (LN && !in.lines_ready) line_values();
#pragma unroll
    for (int j = 0; j < L; j++) {
        rvx[j] = in.own_vx(j);
        rvz[j] = in.own_vz(j);
        rp[j] = in.own_p(j);
    }
#pragma unroll
    for (int q = 0; q < Q::NQX; q++) rhx[q] = th.hx_jj[q] >= 0 ? in.hvx(th.hx_r[q], th.hx_jj[q]) : 0.0f;
#pragma unroll
    for (int q = 0; q < Q::NQZ; q++) rhz[q] = th.hz_kk[q] >= 0 ? in.hvz(th.hz_kk[q], i) : 0.0f;
    // q = C_p pbar over tile + 2k halo
    in.template stage<true>();
    __syncthreads();
    float (&spa)[TZ + 4 * R][TX + 4 * R] = in.sp();

    float qw[W];
#pragma unroll
    for (int w = 0; w < W; w++) qw[w] = spa[rs - R + 1 + w + H][c + H];
#pragma unroll
    for (int j = 0; j < L; j++) {
        const int r = rs + j, k = k0 + r;
        if (LN && a.hbar && colp) {   // transposed pressure injection: hbar[n] = scale sum_k w_k q
            const float w = row_weight(k, a.src.kp, a.src.wp0, a.src.wp1);
            const int jl = i - a.src.i0;
            if (w != 0.0f && jl >= 0 && jl < a.src.n)
                atomicAdd(&a.hbar[(size_t)n * a.src.n + jl],
                          (double)(w * a.src.scale) * (double)qw[j + R - 1]);
        }
        // vbar_x' = vbar_x + D+ q; C_vx vbar_x' kept for the p update
        const bool okx = !SP || (colx && k < NZ);
        const float *row = &spa[r + H][c + H];
        float d = 0.0f;
#pragma unroll
        for (int m = 1; m <= R; m++) d = fmaf(cc[m - 1], row[m] - row[1 - m], d);
        const float vbx = rvx[j] + d;
        float vx, ox;
        if (SP) {
            float A, B;
            damp(sxh + szi[j], A, B);
            vx = okx ? (B * cv) * vbx : 0.0f;
            ox = A * vbx;
        } else {
            vx = cv * vbx;
            ox = vbx;
        }
        if (okx) st_out(io.vx_out + k * pitch + i, ox);
        sm.svx[r][c + R] = vx;
        // vbar_z' likewise, from the window down the column
        const bool okz = !SP || (colp && k < NZ - 1);
        d = 0.0f;
#pragma unroll
        for (int m = 1; m <= R; m++) d = fmaf(cc[m - 1], qw[j + R - 1 + m] - qw[j + R - m], d);
        const float vb = rvz[j] + d;
        float A = 1.0f, B = 1.0f;
        if (SP) damp(sxi + szh[j], A, B);
        float vz = (B * cv) * vb;
        float out = SP ? A * vb : vb;
        if (LN && a.fbar && okz) {   // transposed velocity injection read out
            const float wf = row_weight(k, a.src.kv, a.src.wv0, a.src.wv1);
            const int js = i - a.src.i0;
            if (wf != 0.0f && js >= 0 && js < a.src.n)
                atomicAdd(&a.fbar[(size_t)n * a.src.n + js], (double)(wf * a.src.scale) * (double)vz);
        }
        if (LN && a.yv && n >= 1 && okz) {   // transposed v_z sampling of step n-1
            const float wy_ = row_weight(k, a.rec.kv, a.rec.wv0, a.rec.wv1);
            if (wy_ != 0.0f && jrin) out = fmaf(wy_, yvv, out);
        }
        if (okz) st_out(io.vz_out + k * pitch + i, out);
        sm.svz[r + R][c] = okz ? vz : 0.0f;
    }
    // halo vbar' (not written out)
#pragma unroll
    for (int q = 0; q < Q::NQX; q++) {
        const int jj = th.hx_jj[q], r = th.hx_r[q];
        if (jj < 0) continue;
        const int k = k0 + r, j = i0 - R + jj;
        const float *row = &spa[r + H][jj + R];
        float d = 0.0f;
#pragma unroll
        for (int m = 1; m <= R; m++) d = fmaf(cc[m - 1], row[m] - row[1 - m], d);
        const float vb = rhx[q] + d;
        float val;
        if (SP) {
            const bool ok = k < NZ && j >= 0 && j < NX - 1;
            float A, B;
            damp(__ldg(g.sxh + (ok ? j : 0)) + __ldg(g.szi + (ok ? k : 0)), A, B);
            val = ok ? (B * cv) * vb : 0.0f;
        } else {
            val = cv * vb;
        }
        sm.svx[r][jj] = val;
    }
#pragma unroll
    for (int q = 0; q < Q::NQZ; q++) {
        const int kk = th.hz_kk[q];
        if (kk < 0) continue;
        const int k = k0 - R + kk;
        float d = 0.0f;
#pragma unroll
        for (int m = 1; m <= R; m++)
            d = fmaf(cc[m - 1], spa[kk + R + m][c + H] - spa[kk + R + 1 - m][c + H], d);
        const float vb = rhz[q] + d;
        float val;
        if (SP) {
            const bool ok = colp && k >= 0 && k < NZ - 1;
            float A, B;
            damp(sxi + __ldg(g.szh + (ok ? k : 0)), A, B);
            val = ok ? (B * cv) * vb : 0.0f;
        } else {
            val = (1.0f * cv) * vb;
        }
        sm.svz[kk][c] = val;
    }
    __syncthreads();

    // pbar <- A_p pbar + D- (C_v vbar')
    float zw[W];
#pragma unroll
    for (int w = 0; w < W; w++) zw[w] = sm.svz[rs + w][c];
#pragma unroll
    for (int j = 0; j < L; j++) {
        const int r = rs + j, k = k0 + r;
        const bool okp = !SP || (colp && k < NZ);
        float d = 0.0f;
#pragma unroll
        for (int m = 1; m <= R; m++) {
            d = fmaf(cc[m - 1], sm.svx[r][c + R + m - 1] - sm.svx[r][c + R - m], d);
            d = fmaf(cc[m - 1], zw[j + R + m - 1] - zw[j + R - m], d);
        }
        float out;
        if (SP) {
            float A, B;
            damp(sxi + szi[j], A, B);
            out = fmaf(A, rp[j], d);
        } else {
            out = rp[j] + d;
        }
        if (LN && a.yp && n >= 1 && okp) {   // transposed pressure sampling of step n-1
            const float w = row_weight(k, a.rec.kp, a.rec.wp0, a.rec.wp1);
            if (w != 0.0f && jrin) out = fmaf(w, ypv, out);
        }
        if (okp) st_out(io.p_out + k * pitch + i, out);
    }
}

// ---------------------------------------------------------------------------
// Tiles by quads (order 8). Thread t owns the four consecutive columns
// i0 + c4 .. i0 + c4 + 3, c4 = 4 (t mod TX/4), of tile rows L (t / (TX/4))
// .. + L - 1 (L = 1 or 2 quads down its column, as the CTA size gives). Every
// operand moves as a 16-byte vector: the thread's own v, kappa and p, the x
// differences (the eleven values an 8-point difference of four consecutive
// points needs sit in three aligned quads of a staged row) and the z
// differences (a window of 2k + L - 1 quads down the column, shared by the
// thread's L rows). The halo values of v (2k-1 rows of v_z, a quad of v_x on each side
// of every tile row) are shared out over all threads as quads. Per point the
// arithmetic is the strips' (fwd_strip / adj_strip), term for term and in the
// same order, so every tile configuration still gives the same bits. Tiles
// that a line meets keep the strip step (its injection and sampling).
// ---------------------------------------------------------------------------
template <int R, int TX, int TZ, int NT>
struct QuadShape {
    static constexpr int QW = TX / 4;                      // quads per tile row
    // rows per thread: the thread's quads are rows r .. r + L - 1 of its column
    static constexpr int L = NT > 0 ? TX * TZ / (4 * NT) : 0;
    static constexpr bool ok = R == 4 && TX % 4 == 0 && (L == 1 || L == 2) && NT * 4 * L == TX * TZ;
    static constexpr int NW = 2 * R + L - 1;               // quads of a column window
    static constexpr int NHZ = (2 * R - 1) * QW;           // v_z halo quads
    static constexpr int NHX = 2 * TZ;                     // v_x halo quads
    static constexpr int NH = (NHZ + NHX + NT - 1) / NT;   // halo quads per thread
};

struct Q4 {
    float e[4];
};
__device__ __forceinline__ Q4 q4(const float4 v) { return {{v.x, v.y, v.z, v.w}}; }
__device__ __forceinline__ float4 f4(const Q4 &q) { return make_float4(q.e[0], q.e[1], q.e[2], q.e[3]); }
__device__ __forceinline__ Q4 lds4(const float *p) { return q4(*reinterpret_cast<const float4 *>(p)); }
__device__ __forceinline__ void sts4(float *p, const Q4 &v) { *reinterpret_cast<float4 *>(p) = f4(v); }
__device__ __forceinline__ void st_out4(float *p, const Q4 &v) {
    asm volatile("st.global.cg.v4.f32 [%0], {%1, %2, %3, %4};" ::"l"(p), "f"(v.e[0]), "f"(v.e[1]),
                 "f"(v.e[2]), "f"(v.e[3])
                 : "memory");
}
// a quad of a field into the storage: one vector store where all four points
// are inside the grid, else the points that are (masked points are never written)
__device__ __forceinline__ void st_quad(float *p, const Q4 &v, const bool (&ok)[4], bool all) {
    if (all) {
        st_out4(p, v);
    } else {
#pragma unroll
        for (int e = 0; e < 4; e++)
            if (ok[e]) st_out(p + e, v.e[e]);
    }
}

// the x difference D+ of the four points whose twelve-value window starts at
// x: u[x + e + k + m] - u[x + e + k + 1 - m] (the v_x points of a p row, or
// the p points of a v_x row), accumulated as the strips do
template <int R>
__device__ __forceinline__ Q4 xdiff(const float *x, const float (&cc)[R]) {
    float u[12];
    const Q4 a = lds4(x), b = lds4(x + 4), c = lds4(x + 8);
#pragma unroll
    for (int e = 0; e < 4; e++) {
        u[e] = a.e[e];
        u[4 + e] = b.e[e];
        u[8 + e] = c.e[e];
    }
    Q4 d;
#pragma unroll
    for (int e = 0; e < 4; e++) {
        float s = 0.0f;
#pragma unroll
        for (int m = 1; m <= R; m++) s = fmaf(cc[m - 1], u[e + R + m] - u[e + R + 1 - m], s);
        d.e[e] = s;
    }
    return d;
}
// the z difference of the quad whose 2k-quad column window starts at w[j]:
// w[j + k - 1 + m] - w[j + k - m]
template <int R, int NW>
__device__ __forceinline__ Q4 zdiff(const Q4 (&w)[NW], int j, const float (&cc)[R]) {
    Q4 d;
#pragma unroll
    for (int e = 0; e < 4; e++) {
        float s = 0.0f;
#pragma unroll
        for (int m = 1; m <= R; m++) s = fmaf(cc[m - 1], w[j + R - 1 + m].e[e] - w[j + R - m].e[e], s);
        d.e[e] = s;
    }
    return d;
}
// the NW quads of a column window: rows row0, row0 + 1, ... of a staged field
template <int NW, int PW>
__device__ __forceinline__ void window(Q4 (&w)[NW], const float (*rows)[PW], int row0, int col) {
#pragma unroll
    for (int q = 0; q < NW; q++) w[q] = lds4(&rows[row0 + q][col]);
}

// a thread's quads and its halo items: kind 1 = v_z quad at v_z row a,
// column b; kind 2 = v_x quad at tile row a, v_x column b (x = i0 - k + b);
// kind 0 = none
template <int R, int TX, int TZ, int NT>
struct QuadThread {
    using Q = QuadShape<R, TX, TZ, NT>;
    int c4, r;
    int kind[Q::NH], ha[Q::NH], hb[Q::NH];
    __device__ __forceinline__ QuadThread() {
        const int t = threadIdx.x;
        c4 = 4 * (t % Q::QW);
        r = Q::L * (t / Q::QW);
#pragma unroll
        for (int q = 0; q < Q::NH; q++) {
            const int e = t + q * NT;
            if (e < Q::NHZ) {
                const int hz = e / Q::QW;
                kind[q] = 1;
                ha[q] = hz < R ? hz : hz + TZ;
                hb[q] = 4 * (e % Q::QW);
            } else if (e < Q::NHZ + Q::NHX) {
                const int e2 = e - Q::NHZ;
                kind[q] = 2;
                ha[q] = e2 >> 1;
                hb[q] = (e2 & 1) ? TX + R : 0;
            } else {
                kind[q] = 0;
                ha[q] = hb[q] = 0;
            }
        }
    }
};

// One forward step of a tile by quads (interior or sponge tile; no line).
template <int R, int TX, int TZ, int NT, bool SP, class In, class Work>
__device__ __forceinline__ void fwd_quad(const FwdArgs &a, const StepIO &io, int i0, int k0,
                                         In &in, Work &sm) {
    using Q = QuadShape<R, TX, TZ, NT>;
    constexpr int H = 2 * R, L = Q::L, NW = Q::NW;
    const GridArgs &g = a.g;
    const int pitch = g.pitch, NX = g.NX, NZ = g.NZ;
    const QuadThread<R, TX, TZ, NT> th;
    const int c4 = th.c4, r = th.r, i = i0 + c4, k = k0 + r;
    float cc[R];
#pragma unroll
    for (int m = 0; m < R; m++) cc[m] = g.c[m];
    const float cv = g.cv;

    // the grid's constants before the wait for the previous step, the fields after it
    float sxi[4], sxh[4], szi[L], szh[L];
    if (!In::kAhead) in.wait();
    if (SP) {
#pragma unroll
        for (int e = 0; e < 4; e++) {
            sxi[e] = __ldg(g.sxi + min(i + e, NX - 1));   // clamped: masked points take any value
            sxh[e] = __ldg(g.sxh + min(i + e, NX - 1));
        }
#pragma unroll
        for (int j = 0; j < L; j++) {
            szi[j] = __ldg(g.szi + min(k + j, NZ - 1));
            szh[j] = __ldg(g.szh + min(k + j, NZ - 1));
        }
    }
    Q4 rk[L];
#pragma unroll
    for (int j = 0; j < L; j++) rk[j] = q4(in.kap4(r + j, c4));
    if (In::kAhead) in.wait();
    Q4 rvx[L], rvz[L];
#pragma unroll
    for (int j = 0; j < L; j++) {
        rvx[j] = q4(in.vx4(r + j, c4 + R));
        rvz[j] = q4(in.vz4(r + j + R, c4));
    }
    Q4 rh[Q::NH];
#pragma unroll
    for (int q = 0; q < Q::NH; q++)
        rh[q] = q4(th.kind[q] == 1 ? in.vz4(th.ha[q], th.hb[q])
                                   : th.kind[q] == 2 ? in.vx4(th.ha[q], th.hb[q]) : make_float4(0.f, 0.f, 0.f, 0.f));
    in.template stage<false>();
    if (!In::kStaged) __syncthreads();   // p staged by all threads
    float (&spa)[TZ + 4 * R][TX + 4 * R] = in.sp();

    // own quads: v_z from the column window, v_x from the rows
    Q4 pw[NW];
    window<NW, TX + 4 * R>(pw, spa, r + H - R + 1, c4 + H);
#pragma unroll
    for (int j = 0; j < L; j++) {
        const Q4 d = zdiff<R>(pw, j, cc);
        Q4 vz;
        bool ok[4];
        bool all = true;
#pragma unroll
        for (int e = 0; e < 4; e++) {
            ok[e] = !SP || (i + e < NX && k + j < NZ - 1);
            all = all && ok[e];
            if (SP) {
                float A, B;
                damp(sxi[e] + szh[j], A, B);
                const float cvz = B * cv;
                vz.e[e] = fmaf(-cvz, d.e[e], A * rvz[j].e[e]);
                vz.e[e] = ok[e] ? vz.e[e] : 0.0f;
            } else {
                vz.e[e] = fmaf(-cv, d.e[e], rvz[j].e[e]);
            }
        }
        st_quad(io.vz_out + (k + j) * pitch + i, vz, ok, all);
        sts4(&sm.svz[r + j + R][c4], vz);
    }
#pragma unroll
    for (int j = 0; j < L; j++) {
        const Q4 d = xdiff<R>(&spa[r + j + H][c4 + R], cc);
        Q4 vx;
        bool ok[4];
        bool all = true;
#pragma unroll
        for (int e = 0; e < 4; e++) {
            ok[e] = !SP || (i + e < NX - 1 && k + j < NZ);
            all = all && ok[e];
            if (SP) {
                float A, B;
                damp(sxh[e] + szi[j], A, B);
                vx.e[e] = fmaf(-(B * cv), d.e[e], A * rvx[j].e[e]);
                vx.e[e] = ok[e] ? vx.e[e] : 0.0f;
            } else {
                vx.e[e] = fmaf(-cv, d.e[e], rvx[j].e[e]);
            }
        }
        st_quad(io.vx_out + (k + j) * pitch + i, vx, ok, all);
        sts4(&sm.svx[r + j][c4 + R], vx);
    }
    Q4 pold[L];
#pragma unroll
    for (int j = 0; j < L; j++) pold[j] = pw[j + R - 1];
    // halo v (not written out)
#pragma unroll
    for (int q = 0; q < Q::NH; q++) {
        const int ha = th.ha[q], hb = th.hb[q];
        if (th.kind[q] == 1) {
            const int kh = k0 - R + ha;
            Q4 w[2 * R];
            window<2 * R, TX + 4 * R>(w, spa, ha + 1, hb + H);
            const Q4 d = zdiff<R>(w, 0, cc);
            Q4 val;
#pragma unroll
            for (int e = 0; e < 4; e++) {
                if (SP) {
                    const int ih = i0 + hb + e;
                    const bool ok = ih < NX && kh >= 0 && kh < NZ - 1;
                    float A, B;
                    damp(__ldg(g.sxi + min(ih, NX - 1)) + __ldg(g.szh + (ok ? kh : 0)), A, B);
                    const float cvz = B * cv;
                    const float v = fmaf(-cvz, d.e[e], A * rh[q].e[e]);
                    val.e[e] = ok ? v : 0.0f;
                } else {
                    val.e[e] = fmaf(-cv, d.e[e], rh[q].e[e]);
                }
            }
            sts4(&sm.svz[ha][hb], val);
        } else if (th.kind[q] == 2) {
            const int kh = k0 + ha;
            const Q4 d = xdiff<R>(&spa[ha + H][hb], cc);
            Q4 val;
#pragma unroll
            for (int e = 0; e < 4; e++) {
                if (SP) {
                    const int j = i0 - R + hb + e;
                    const bool ok = kh < NZ && j >= 0 && j < NX - 1;
                    float A, B;
                    damp(__ldg(g.sxh + (ok ? j : 0)) + __ldg(g.szi + (ok ? kh : 0)), A, B);
                    val.e[e] = ok ? fmaf(-(B * cv), d.e[e], A * rh[q].e[e]) : 0.0f;
                } else {
                    val.e[e] = fmaf(-cv, d.e[e], rh[q].e[e]);
                }
            }
            sts4(&sm.svx[ha][hb], val);
        }
    }
    __syncthreads();

    // own quads: p^{n+1}, z differences from a window over the v_z rows
    Q4 zw[NW];
    window<NW, TX>(zw, sm.svz, r, c4);
#pragma unroll
    for (int j = 0; j < L; j++) {
        float u[12];
        {
            const Q4 a0 = lds4(&sm.svx[r + j][c4]), a1 = lds4(&sm.svx[r + j][c4 + 4]),
                     a2 = lds4(&sm.svx[r + j][c4 + 8]);
#pragma unroll
            for (int e = 0; e < 4; e++) {
                u[e] = a0.e[e];
                u[4 + e] = a1.e[e];
                u[8 + e] = a2.e[e];
            }
        }
        Q4 val;
        bool ok[4];
        bool all = true;
#pragma unroll
        for (int e = 0; e < 4; e++) {
            float d = 0.0f;
#pragma unroll
            for (int m = 1; m <= R; m++) {
                d = fmaf(cc[m - 1], u[e + R + m - 1] - u[e + R - m], d);
                d = fmaf(cc[m - 1], zw[j + R + m - 1].e[e] - zw[j + R - m].e[e], d);
            }
            ok[e] = !SP || (i + e < NX && k + j < NZ);
            all = all && ok[e];
            float cp = rk[j].e[e];
            if (SP) {
                float A, B;
                damp(sxi[e] + szi[j], A, B);
                cp *= B;
                val.e[e] = fmaf(-cp, d, A * pold[j].e[e]);
            } else {
                val.e[e] = fmaf(-cp, d, pold[j].e[e]);
            }
        }
        st_quad(io.p_out + (k + j) * pitch + i, val, ok, all);
    }
}

// One transposed step of a tile by quads (interior or sponge tile; no line).
template <int R, int TX, int TZ, int NT, bool SP, class In, class Work>
__device__ __forceinline__ void adj_quad(const AdjArgs &a, const StepIO &io, int i0, int k0,
                                         In &in, Work &sm) {
    using Q = QuadShape<R, TX, TZ, NT>;
    constexpr int H = 2 * R, L = Q::L, NW = Q::NW;
    const GridArgs &g = a.g;
    const int pitch = g.pitch, NX = g.NX, NZ = g.NZ;
    const QuadThread<R, TX, TZ, NT> th;
    const int c4 = th.c4, r = th.r, i = i0 + c4, k = k0 + r;
    float cc[R];
#pragma unroll
    for (int m = 0; m < R; m++) cc[m] = g.c[m];
    const float cv = g.cv;

    float sxi[4], sxh[4], szi[L], szh[L];
    if (!In::kAhead) in.wait();
    if (SP) {
#pragma unroll
        for (int e = 0; e < 4; e++) {
            sxi[e] = __ldg(g.sxi + min(i + e, NX - 1));
            sxh[e] = __ldg(g.sxh + min(i + e, NX - 1));
        }
#pragma unroll
        for (int j = 0; j < L; j++) {
            szi[j] = __ldg(g.szi + min(k + j, NZ - 1));
            szh[j] = __ldg(g.szh + min(k + j, NZ - 1));
        }
    }
    in.template prestage<true>();   // C_p of the staged region (constants)
    if (In::kAhead) in.wait();
    Q4 rvx[L], rvz[L], rp[L];
#pragma unroll
    for (int j = 0; j < L; j++) {
        rvx[j] = q4(in.vx4(r + j, c4 + R));
        rvz[j] = q4(in.vz4(r + j + R, c4));
        rp[j] = q4(in.p4(r + j, c4));
    }
    Q4 rh[Q::NH];
#pragma unroll
    for (int q = 0; q < Q::NH; q++)
        rh[q] = q4(th.kind[q] == 1 ? in.vz4(th.ha[q], th.hb[q])
                                   : th.kind[q] == 2 ? in.vx4(th.ha[q], th.hb[q]) : make_float4(0.f, 0.f, 0.f, 0.f));
    // q = C_p pbar over tile + 2k halo
    in.template stage<true>();
    __syncthreads();
    float (&spa)[TZ + 4 * R][TX + 4 * R] = in.sp();

#pragma unroll
    for (int j = 0; j < L; j++) {   // vbar_x' = vbar_x + D+ q; C_vx vbar_x' kept for the p update
        const Q4 d = xdiff<R>(&spa[r + j + H][c4 + R], cc);
        Q4 vx, ox;
        bool ok[4];
        bool all = true;
#pragma unroll
        for (int e = 0; e < 4; e++) {
            ok[e] = !SP || (i + e < NX - 1 && k + j < NZ);
            all = all && ok[e];
            const float vbx = rvx[j].e[e] + d.e[e];
            if (SP) {
                float A, B;
                damp(sxh[e] + szi[j], A, B);
                vx.e[e] = ok[e] ? (B * cv) * vbx : 0.0f;
                ox.e[e] = A * vbx;
            } else {
                vx.e[e] = cv * vbx;
                ox.e[e] = vbx;
            }
        }
        st_quad(io.vx_out + (k + j) * pitch + i, ox, ok, all);
        sts4(&sm.svx[r + j][c4 + R], vx);
    }
    {   // vbar_z' likewise, from the window down the column
        Q4 w[NW];
        window<NW, TX + 4 * R>(w, spa, r + H - R + 1, c4 + H);
#pragma unroll
        for (int j = 0; j < L; j++) {
            const Q4 d = zdiff<R>(w, j, cc);
            Q4 vz, out;
            bool ok[4];
            bool all = true;
#pragma unroll
            for (int e = 0; e < 4; e++) {
                ok[e] = !SP || (i + e < NX && k + j < NZ - 1);
                all = all && ok[e];
                const float vb = rvz[j].e[e] + d.e[e];
                float A = 1.0f, B = 1.0f;
                if (SP) damp(sxi[e] + szh[j], A, B);
                const float v = (B * cv) * vb;
                out.e[e] = SP ? A * vb : vb;
                vz.e[e] = ok[e] ? v : 0.0f;
            }
            st_quad(io.vz_out + (k + j) * pitch + i, out, ok, all);
            sts4(&sm.svz[r + j + R][c4], vz);
        }
    }
    // halo vbar' (not written out)
#pragma unroll
    for (int q = 0; q < Q::NH; q++) {
        const int ha = th.ha[q], hb = th.hb[q];
        if (th.kind[q] == 1) {
            const int kh = k0 - R + ha;
            Q4 w[2 * R];
            window<2 * R, TX + 4 * R>(w, spa, ha + 1, hb + H);
            const Q4 d = zdiff<R>(w, 0, cc);
            Q4 val;
#pragma unroll
            for (int e = 0; e < 4; e++) {
                const float vb = rh[q].e[e] + d.e[e];
                if (SP) {
                    const int ih = i0 + hb + e;
                    const bool ok = ih < NX && kh >= 0 && kh < NZ - 1;
                    float A, B;
                    damp(__ldg(g.sxi + min(ih, NX - 1)) + __ldg(g.szh + (ok ? kh : 0)), A, B);
                    val.e[e] = ok ? (B * cv) * vb : 0.0f;
                } else {
                    val.e[e] = (1.0f * cv) * vb;
                }
            }
            sts4(&sm.svz[ha][hb], val);
        } else if (th.kind[q] == 2) {
            const int kh = k0 + ha;
            const Q4 d = xdiff<R>(&spa[ha + H][hb], cc);
            Q4 val;
#pragma unroll
            for (int e = 0; e < 4; e++) {
                const float vb = rh[q].e[e] + d.e[e];
                if (SP) {
                    const int j = i0 - R + hb + e;
                    const bool ok = kh < NZ && j >= 0 && j < NX - 1;
                    float A, B;
                    damp(__ldg(g.sxh + (ok ? j : 0)) + __ldg(g.szi + (ok ? kh : 0)), A, B);
                    val.e[e] = ok ? (B * cv) * vb : 0.0f;
                } else {
                    val.e[e] = cv * vb;
                }
            }
            sts4(&sm.svx[ha][hb], val);
        }
    }
    __syncthreads();

    // pbar <- A_p pbar + D- (C_v vbar')
    Q4 zw[NW];
    window<NW, TX>(zw, sm.svz, r, c4);
#pragma unroll
    for (int j = 0; j < L; j++) {
        float u[12];
        {
            const Q4 a0 = lds4(&sm.svx[r + j][c4]), a1 = lds4(&sm.svx[r + j][c4 + 4]),
                     a2 = lds4(&sm.svx[r + j][c4 + 8]);
#pragma unroll
            for (int e = 0; e < 4; e++) {
                u[e] = a0.e[e];
                u[4 + e] = a1.e[e];
                u[8 + e] = a2.e[e];
            }
        }
        Q4 out;
        bool ok[4];
        bool all = true;
#pragma unroll
        for (int e = 0; e < 4; e++) {
            float d = 0.0f;
#pragma unroll
            for (int m = 1; m <= R; m++) {
                d = fmaf(cc[m - 1], u[e + R + m - 1] - u[e + R - m], d);
                d = fmaf(cc[m - 1], zw[j + R + m - 1].e[e] - zw[j + R - m].e[e], d);
            }
            ok[e] = !SP || (i + e < NX && k + j < NZ);
            all = all && ok[e];
            if (SP) {
                float A, B;
                damp(sxi[e] + szi[j], A, B);
                out.e[e] = fmaf(A, rp[j].e[e], d);
            } else {
                out.e[e] = rp[j].e[e] + d;
            }
        }
        st_quad(io.p_out + (k + j) * pitch + i, out, ok, all);
    }
}

// V = 1: interior and sponge tiles step by quads where the shape allows it
// (QuadShape::ok), tiles that a line meets by strips; V = 0: all by strips.
template <int R, int TX, int TZ, int NT, int V = 0>
__device__ __forceinline__ void fwd_tile(const FwdArgs &a, const StepIO &io, int i0, int k0,
                                         TileSmem<R, TX, TZ> &sm, bool lines_ready = false) {
    const bool in = interior_tile<R, TX, TZ>(a.g, i0, k0);
    if constexpr (StripShape<R, TX, TZ, NT>::ok) {
        using Q = StripShape<R, TX, TZ, NT>;
        constexpr bool kQuads = V == 1 && QuadShape<R, TX, TZ, NT>::ok;
        const int c = threadIdx.x % TX, rs = (threadIdx.x / TX) * Q::L;
        // three variants: interior tiles, sponge / edge tiles, and tiles a line
        // meets (the general one, which reduces to the same arithmetic where a
        // point is undamped and inside the grid)
        if (fwd_lines<R, TZ>(a, k0)) {
            GlobalIn<R, TX, TZ, NT, true> gi(a.g, io, i0, k0, rs, c, sm, lines_ready);
            fwd_strip<R, TX, TZ, NT, true, true>(a, io, i0, k0, gi, sm);
        } else if (in) {
            GlobalIn<R, TX, TZ, NT, false> gi(a.g, io, i0, k0, rs, c, sm, lines_ready);
            if constexpr (kQuads) fwd_quad<R, TX, TZ, NT, false>(a, io, i0, k0, gi, sm);
            else fwd_strip<R, TX, TZ, NT, false, false>(a, io, i0, k0, gi, sm);
        } else {
            GlobalIn<R, TX, TZ, NT, true> gi(a.g, io, i0, k0, rs, c, sm, lines_ready);
            if constexpr (kQuads) fwd_quad<R, TX, TZ, NT, true>(a, io, i0, k0, gi, sm);
            else fwd_strip<R, TX, TZ, NT, true, false>(a, io, i0, k0, gi, sm);
        }
    } else {
        if (in) fwd_tile_impl<R, TX, TZ, NT, false>(a, io, i0, k0, sm);
        else fwd_tile_impl<R, TX, TZ, NT, true>(a, io, i0, k0, sm);
    }
}

template <int R, int TX, int TZ, int NT, int V = 0>
__device__ __forceinline__ void adj_tile(const AdjArgs &a, const StepIO &io, int i0, int k0,
                                         TileSmem<R, TX, TZ> &sm, bool lines_ready = false) {
    const bool in = interior_tile<R, TX, TZ>(a.g, i0, k0);
    if constexpr (StripShape<R, TX, TZ, NT>::ok) {
        using Q = StripShape<R, TX, TZ, NT>;
        constexpr bool kQuads = V == 1 && QuadShape<R, TX, TZ, NT>::ok;
        const int c = threadIdx.x % TX, rs = (threadIdx.x / TX) * Q::L;
        // three variants: interior tiles, sponge / edge tiles, and tiles a line
        // meets (the general one, which reduces to the same arithmetic where a
        // point is undamped and inside the grid)
        if (adj_lines<TZ>(a, k0, io.n)) {
            GlobalIn<R, TX, TZ, NT, true> gi(a.g, io, i0, k0, rs, c, sm, lines_ready);
            adj_strip<R, TX, TZ, NT, true, true>(a, io, i0, k0, gi, sm);
        } else if (in) {
            GlobalIn<R, TX, TZ, NT, false> gi(a.g, io, i0, k0, rs, c, sm, lines_ready);
            if constexpr (kQuads) adj_quad<R, TX, TZ, NT, false>(a, io, i0, k0, gi, sm);
            else adj_strip<R, TX, TZ, NT, false, false>(a, io, i0, k0, gi, sm);
        } else {
            GlobalIn<R, TX, TZ, NT, true> gi(a.g, io, i0, k0, rs, c, sm, lines_ready);
            if constexpr (kQuads) adj_quad<R, TX, TZ, NT, true>(a, io, i0, k0, gi, sm);
            else adj_strip<R, TX, TZ, NT, true, false>(a, io, i0, k0, gi, sm);
        }
    } else {
        if (in) adj_tile_impl<R, TX, TZ, NT, false>(a, io, i0, k0, sm);
        else adj_tile_impl<R, TX, TZ, NT, true>(a, io, i0, k0, sm);
    }
}

// Resident CTAs per SM that the register budget is sized for: a step's tiles
// should fit in one wave (152 SMs x 3 CTAs of 256 threads covers the 418
// tiles of a 681 x 381 grid and its two slabs).
// Strips of 8 or more rows need more registers: two CTAs of 256 threads.
constexpr int min_ctas(int nt, int rows_per_thread = 4) {
    return nt <= 256 ? (rows_per_thread >= 8 ? 2 : 3) : nt <= 512 ? 2 : 1;
}
template <int TX, int TZ, int NT>
constexpr int tile_min_ctas() { return min_ctas(NT, NT >= TX ? TZ / (NT / TX) : 1); }

template <int R, int TX, int TZ>
__device__ __forceinline__ TileSmem<R, TX, TZ> &tile_smem() {
    extern __shared__ __align__(16) unsigned char ssx_smem[];
    return *reinterpret_cast<TileSmem<R, TX, TZ> *>(ssx_smem);
}

template <int R, int TX, int TZ, int NT, int V>
__global__ void __launch_bounds__(NT, (tile_min_ctas<TX, TZ, NT>())) k_fwd(const FwdArgs a) {
    griddep_launch();   // the tile step waits for the previous step itself
    const StepIO io{a.p_in, a.vx_in, a.vz_in, a.p_out, a.vx_out, a.vz_out, a.n};
    fwd_tile<R, TX, TZ, NT, V>(a, io, blockIdx.x * TX, blockIdx.y * TZ, tile_smem<R, TX, TZ>());
}

template <int R, int TX, int TZ, int NT, int V>
__global__ void __launch_bounds__(NT, (tile_min_ctas<TX, TZ, NT>())) k_adj(const AdjArgs a) {
    griddep_launch();
    const StepIO io{a.p_in, a.vx_in, a.vz_in, a.p_out, a.vx_out, a.vz_out, a.n};
    adj_tile<R, TX, TZ, NT, V>(a, io, blockIdx.x * TX, blockIdx.y * TZ, tile_smem<R, TX, TZ>());
}

// ---------------------------------------------------------------------------
// Persistent sweep: one cooperative launch runs all nt steps. CTA b owns tile
// b for the whole sweep. Before step n it waits until its four edge
// neighbours have published "n steps done" (their step n-1 outputs, which
// its halo reads, are complete, and they no longer read the buffer it is
// about to overwrite); after the step it publishes n+1. The tile is at least
// 2k wide in both directions, so the halo never reaches beyond those four
// neighbours. Waits are bounded: past `timeout_ns` of %globaltimer the CTA
// records an error and every CTA leaves the sweep.
// ---------------------------------------------------------------------------
__device__ __forceinline__ unsigned ld_acquire(const unsigned *p) {
    unsigned v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ void st_release(unsigned *p, unsigned v) {
    asm volatile("st.release.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}
__device__ __forceinline__ unsigned long long globaltimer() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %globaltimer;" : "=l"(t));
    return t;
}

// true = go on; false = leave the sweep (timeout here or elsewhere)
__device__ __forceinline__ bool wait_neighbours(const PersistArgs &pa, int tile, unsigned need,
                                                int *s_abort) {
    if (threadIdx.x < 4) {
        const int tx = tile % pa.tiles_x, tz = tile / pa.tiles_x;
        int nb = -1;
        if (threadIdx.x == 0 && tx > 0) nb = tile - 1;
        if (threadIdx.x == 1 && tx + 1 < pa.tiles_x) nb = tile + 1;
        if (threadIdx.x == 2 && tz > 0) nb = tile - pa.tiles_x;
        if (threadIdx.x == 3 && tz + 1 < pa.tiles_z) nb = tile + pa.tiles_x;
        if (nb >= 0 && ld_acquire(pa.flags + nb) < need) {
            const unsigned long long t0 = globaltimer();
            unsigned spins = 0;
            while (ld_acquire(pa.flags + nb) < need) {
                if ((++spins & 63u) == 0) {
                    if (*(volatile int *)pa.err != 0) {
                        *s_abort = 1;
                        break;
                    }
                    if (globaltimer() - t0 > pa.timeout_ns) {
                        atomicExch(pa.err, 1);
                        *s_abort = 1;
                        break;
                    }
                }
                __nanosleep(20);
            }
        }
    }
    __syncthreads();
    return *s_abort == 0;
}

__device__ __forceinline__ void publish(const PersistArgs &pa, int tile, unsigned done) {
    __syncthreads();
    if (threadIdx.x == 0 && tile != pa.stall_tile) {
        __threadfence();
        st_release(pa.flags + tile, done);
    }
}

// step io of a ping-pong sweep: even steps read buffer 0, odd steps buffer 1
__device__ __forceinline__ StepIO ping_pong(const PersistArgs &pa, int t, int n) {
    const bool odd = t & 1;
    StepIO io;
    io.p_in = odd ? pa.f[1][0] : pa.f[0][0];
    io.vx_in = odd ? pa.f[1][1] : pa.f[0][1];
    io.vz_in = odd ? pa.f[1][2] : pa.f[0][2];
    io.p_out = odd ? pa.f[0][0] : pa.f[1][0];
    io.vx_out = odd ? pa.f[0][1] : pa.f[1][1];
    io.vz_out = odd ? pa.f[0][2] : pa.f[1][2];
    io.n = n;
    return io;
}

template <int R, int TX, int TZ, int NT, int V>
__global__ void __launch_bounds__(NT) k_fwd_persist(const FwdArgs a, const PersistArgs pa) {
    TileSmem<R, TX, TZ> &sm = tile_smem<R, TX, TZ>();
    __shared__ int s_abort;
    if (threadIdx.x == 0) s_abort = 0;
    __syncthreads();
    const int tile = blockIdx.x;
    const int i0 = (tile % pa.tiles_x) * TX, k0 = (tile / pa.tiles_x) * TZ;
    for (int n = 0; n < pa.nt; n++) {
        if (n > 0 && !wait_neighbours(pa, tile, (unsigned)n, &s_abort)) return;
        fwd_tile<R, TX, TZ, NT, V>(a, ping_pong(pa, n, n), i0, k0, sm);
        publish(pa, tile, (unsigned)(n + 1));
    }
}

template <int R, int TX, int TZ, int NT, int V>
__global__ void __launch_bounds__(NT) k_adj_persist(const AdjArgs a, const PersistArgs pa) {
    TileSmem<R, TX, TZ> &sm = tile_smem<R, TX, TZ>();
    __shared__ int s_abort;
    if (threadIdx.x == 0) s_abort = 0;
    __syncthreads();
    const int tile = blockIdx.x;
    const int i0 = (tile % pa.tiles_x) * TX, k0 = (tile / pa.tiles_x) * TZ;
    for (int t = 0; t < pa.nt; t++) {
        if (t > 0 && !wait_neighbours(pa, tile, (unsigned)t, &s_abort)) return;
        adj_tile<R, TX, TZ, NT, V>(a, ping_pong(pa, t, pa.nt - 1 - t), i0, k0, sm);
        publish(pa, tile, (unsigned)(t + 1));
    }
}

// One time step of every sweep of a phase (launch t). The sweeps arrive as
// the kernel parameter; the CTA finds its sweep and steps its tile if that
// sweep is active in this launch.
// ONE: the phase has a single sweep, so its arguments sit at fixed offsets of
// the parameter bank and the step reads them as constant operands instead of
// loading them through a runtime sweep index.
template <int R, int TX, int TZ, int NT, int V, bool ONE>
__global__ void __launch_bounds__(NT, (tile_min_ctas<TX, TZ, NT>())) k_multi(const JobSet P, int t) {
    griddep_launch();
    int j = 0;
    if (!ONE) {
#pragma unroll
        for (int q = 1; q < kMaxJobs; q++)
            if (q < P.njobs && (int)blockIdx.x >= P.job[q].tile_base) j = q;
    }
    const Job &J = P.job[j];
    const int st = t - J.offset;
    if (st < 0 || st >= J.nt) return;
    int i0, k0;
    tile_corner<TX, TZ>(J.tx_mul, J.tx_shift, J.tiles_x, blockIdx.x - J.tile_base, i0, k0);
    const bool odd = st & 1;
    StepIO io;
    io.p_in = odd ? J.f[1][0] : J.f[0][0];
    io.vx_in = odd ? J.f[1][1] : J.f[0][1];
    io.vz_in = odd ? J.f[1][2] : J.f[0][2];
    io.p_out = odd ? J.f[0][0] : J.f[1][0];
    io.vx_out = odd ? J.f[0][1] : J.f[1][1];
    io.vz_out = odd ? J.f[0][2] : J.f[1][2];
    io.n = J.adj ? J.nt - 1 - st : st;
    // the tile step reads the grid's constants, then waits for the previous
    // step (griddepcontrol.wait) before its field loads
    // a sweep that starts with the phase injects gathers made before it:
    // its line values are read before the wait too (the phase's first
    // launch is not a dependent launch, so everything before it is complete)
    if (J.adj)
        adj_tile<R, TX, TZ, NT, V>(J.aa, io, i0, k0, tile_smem<R, TX, TZ>(), J.offset == 0);
    else
        fwd_tile<R, TX, TZ, NT, V>(J.fa, io, i0, k0, tile_smem<R, TX, TZ>(), J.offset == 0);
}

// The same for a phase whose sweeps live in a device table (batches of many
// shots, each launch streams far more data than the look-up costs): binary
// search of the CTA's sweep, its arguments copied to shared memory.
template <int R, int TX, int TZ, int NT, int V>
__global__ void __launch_bounds__(NT, (tile_min_ctas<TX, TZ, NT>())) k_multi_tab(const Job *__restrict__ jobs, int njobs, int t) {
    griddep_launch();
    __shared__ Job sj;
    __shared__ int s_j;
    if (threadIdx.x == 0) {
        int lo = 0, hi = njobs - 1;
        while (lo < hi) {   // last sweep whose tile_base <= blockIdx.x
            const int mid = (lo + hi + 1) >> 1;
            if (__ldg(&jobs[mid].tile_base) <= (int)blockIdx.x) lo = mid; else hi = mid - 1;
        }
        s_j = lo;
    }
    __syncthreads();
    {
        const int *src = reinterpret_cast<const int *>(jobs + s_j);
        int *dst = reinterpret_cast<int *>(&sj);
        for (int w = threadIdx.x; w < (int)(sizeof(Job) / sizeof(int)); w += NT) dst[w] = __ldg(src + w);
    }
    __syncthreads();
    const int st = t - sj.offset;
    if (st < 0 || st >= sj.nt) return;
    int i0, k0;
    tile_corner<TX, TZ>(sj.tx_mul, sj.tx_shift, sj.tiles_x, blockIdx.x - sj.tile_base, i0, k0);
    const bool odd = st & 1;
    StepIO io;
    io.p_in = odd ? sj.f[1][0] : sj.f[0][0];
    io.vx_in = odd ? sj.f[1][1] : sj.f[0][1];
    io.vz_in = odd ? sj.f[1][2] : sj.f[0][2];
    io.p_out = odd ? sj.f[0][0] : sj.f[1][0];
    io.vx_out = odd ? sj.f[0][1] : sj.f[1][1];
    io.vz_out = odd ? sj.f[0][2] : sj.f[1][2];
    io.n = sj.adj ? sj.nt - 1 - st : st;
    // batches of many shots are bound by throughput, not by the step's
    // latency: wait here (the tile step's own wait is then a no-op)
    griddep_wait();
    if (sj.adj)
        adj_tile<R, TX, TZ, NT, V>(sj.aa, io, i0, k0, tile_smem<R, TX, TZ>());
    else
        fwd_tile<R, TX, TZ, NT, V>(sj.fa, io, i0, k0, tile_smem<R, TX, TZ>());
}

// ----------------------------------------------------------- launchers --
template <int R>
struct Stencil {
    template <int TX, int TZ>
    static size_t smem() { return sizeof(TileSmem<R, TX, TZ>); }

    template <class Args>
    static cudaError_t launch(void (*kern)(Args), dim3 grid, int nt, size_t sm, cudaStream_t s,
                              bool pdl, const Args &a) {
        cudaLaunchConfig_t cfg = {};
        cfg.gridDim = grid;
        cfg.blockDim = dim3(nt);
        cfg.dynamicSmemBytes = sm;
        cfg.stream = s;
        cudaLaunchAttribute at[1];
        at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
        at[0].val.programmaticStreamSerializationAllowed = 1;
        cfg.attrs = pdl ? at : nullptr;
        cfg.numAttrs = pdl ? 1 : 0;
        return cudaLaunchKernelEx(&cfg, kern, a);
    }

    template <int TX, int TZ, int NT, int V>
    static cudaError_t fwd_step(const FwdArgs &a, cudaStream_t s, bool pdl) {
        dim3 grid((a.g.NX + TX - 1) / TX, (a.g.NZ + TZ - 1) / TZ);
        return launch<FwdArgs>(k_fwd<R, TX, TZ, NT, V>, grid, NT, smem<TX, TZ>(), s, pdl, a);
    }
    template <int TX, int TZ, int NT, int V>
    static cudaError_t adj_step(const AdjArgs &a, cudaStream_t s, bool pdl) {
        dim3 grid((a.g.NX + TX - 1) / TX, (a.g.NZ + TZ - 1) / TZ);
        return launch<AdjArgs>(k_adj<R, TX, TZ, NT, V>, grid, NT, smem<TX, TZ>(), s, pdl, a);
    }
    template <int TX, int TZ, int NT, int V>
    static cudaError_t multi(const JobSet &jobs, int total, int t, cudaStream_t s, bool pdl) {
        cudaLaunchConfig_t cfg = {};
        cfg.gridDim = dim3(total);
        cfg.blockDim = dim3(NT);
        cfg.dynamicSmemBytes = smem<TX, TZ>();
        cfg.stream = s;
        cudaLaunchAttribute at[1];
        at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
        at[0].val.programmaticStreamSerializationAllowed = 1;
        cfg.attrs = pdl ? at : nullptr;
        cfg.numAttrs = pdl ? 1 : 0;
        if (jobs.njobs == 1) return cudaLaunchKernelEx(&cfg, k_multi<R, TX, TZ, NT, V, true>, jobs, t);
        return cudaLaunchKernelEx(&cfg, k_multi<R, TX, TZ, NT, V, false>, jobs, t);
    }
    template <int TX, int TZ, int NT, int V>
    static cudaError_t multi_tab(const Job *jobs, int njobs, int total, int t, cudaStream_t s,
                                 bool pdl) {
        cudaLaunchConfig_t cfg = {};
        cfg.gridDim = dim3(total);
        cfg.blockDim = dim3(NT);
        cfg.dynamicSmemBytes = smem<TX, TZ>();
        cfg.stream = s;
        cudaLaunchAttribute at[1];
        at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
        at[0].val.programmaticStreamSerializationAllowed = 1;
        cfg.attrs = pdl ? at : nullptr;
        cfg.numAttrs = pdl ? 1 : 0;
        return cudaLaunchKernelEx(&cfg, k_multi_tab<R, TX, TZ, NT, V>, jobs, njobs, t);
    }
    template <int TX, int TZ, int NT, int V>
    static cudaError_t fwd_persist(const FwdArgs &a, const PersistArgs &pa, cudaStream_t s) {
        FwdArgs aa = a;
        PersistArgs pp = pa;
        void *args[] = {&aa, &pp};
        return cudaLaunchCooperativeKernel((void *)k_fwd_persist<R, TX, TZ, NT, V>,
                                           dim3(pa.tiles_x * pa.tiles_z), dim3(NT), args,
                                           smem<TX, TZ>(), s);
    }
    template <int TX, int TZ, int NT, int V>
    static cudaError_t adj_persist(const AdjArgs &a, const PersistArgs &pa, cudaStream_t s) {
        AdjArgs aa = a;
        PersistArgs pp = pa;
        void *args[] = {&aa, &pp};
        return cudaLaunchCooperativeKernel((void *)k_adj_persist<R, TX, TZ, NT, V>,
                                           dim3(pa.tiles_x * pa.tiles_z), dim3(NT), args,
                                           smem<TX, TZ>(), s);
    }
    template <int TX, int TZ, int NT, int V>
    static cudaError_t prepare() {
        const int sm = (int)smem<TX, TZ>();
        cudaError_t e;
        if ((e = cudaFuncSetAttribute(k_fwd<R, TX, TZ, NT, V>, cudaFuncAttributeMaxDynamicSharedMemorySize, sm)) != cudaSuccess) return e;
        if ((e = cudaFuncSetAttribute(k_adj<R, TX, TZ, NT, V>, cudaFuncAttributeMaxDynamicSharedMemorySize, sm)) != cudaSuccess) return e;
        if ((e = cudaFuncSetAttribute(k_fwd_persist<R, TX, TZ, NT, V>, cudaFuncAttributeMaxDynamicSharedMemorySize, sm)) != cudaSuccess) return e;
        if ((e = cudaFuncSetAttribute(k_multi<R, TX, TZ, NT, V, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, sm)) != cudaSuccess) return e;
        if ((e = cudaFuncSetAttribute(k_multi<R, TX, TZ, NT, V, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, sm)) != cudaSuccess) return e;
        if ((e = cudaFuncSetAttribute(k_multi_tab<R, TX, TZ, NT, V>, cudaFuncAttributeMaxDynamicSharedMemorySize, sm)) != cudaSuccess) return e;
        return cudaFuncSetAttribute(k_adj_persist<R, TX, TZ, NT, V>, cudaFuncAttributeMaxDynamicSharedMemorySize, sm);
    }
    template <int TX, int TZ, int NT, int V>
    static int capacity(bool adj) {
        int dev = 0, sms = 0, per_sm = 0, coop = 0;
        if (cudaGetDevice(&dev) != cudaSuccess) return 0;
        if (cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, dev) != cudaSuccess || !coop) return 0;
        if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return 0;
        const void *fn = adj ? (const void *)k_adj_persist<R, TX, TZ, NT, V> : (const void *)k_fwd_persist<R, TX, TZ, NT, V>;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, NT, smem<TX, TZ>()) != cudaSuccess) return 0;
        return per_sm * sms;
    }
};

}  // namespace

// Dispatch over kTileCfgs for one R (defines stencil_*_r<R> of ssx_internal.cuh).
#define SSX_DEFINE_DISPATCH(RR)                                                                    \
    cudaError_t stencil_fwd_step_r##RR(const FwdArgs &a, int cfg, cudaStream_t s, bool pdl) {      \
        switch (cfg) {                                                                             \
            SSX_TILE_CONFIGS(SSX_CASE_FWD_STEP)                                                    \
            default: return cudaErrorInvalidValue;                                                 \
        }                                                                                          \
    }                                                                                              \
    cudaError_t stencil_adj_step_r##RR(const AdjArgs &a, int cfg, cudaStream_t s, bool pdl) {      \
        switch (cfg) {                                                                             \
            SSX_TILE_CONFIGS(SSX_CASE_ADJ_STEP)                                                    \
            default: return cudaErrorInvalidValue;                                                 \
        }                                                                                          \
    }                                                                                              \
    cudaError_t stencil_fwd_persist_r##RR(const FwdArgs &a, const PersistArgs &pa, int cfg,        \
                                          cudaStream_t s) {                                        \
        switch (cfg) {                                                                             \
            SSX_TILE_CONFIGS(SSX_CASE_FWD_PERSIST)                                                 \
            default: return cudaErrorInvalidValue;                                                 \
        }                                                                                          \
    }                                                                                              \
    cudaError_t stencil_adj_persist_r##RR(const AdjArgs &a, const PersistArgs &pa, int cfg,        \
                                          cudaStream_t s) {                                        \
        switch (cfg) {                                                                             \
            SSX_TILE_CONFIGS(SSX_CASE_ADJ_PERSIST)                                                 \
            default: return cudaErrorInvalidValue;                                                 \
        }                                                                                          \
    }                                                                                              \
    cudaError_t stencil_multi_r##RR(const JobSet &jobs, int total, int t, int cfg, cudaStream_t s, \
                                    bool pdl) {                                                    \
        switch (cfg) {                                                                             \
            SSX_TILE_CONFIGS(SSX_CASE_MULTI)                                                       \
            default: return cudaErrorInvalidValue;                                                 \
        }                                                                                          \
    }                                                                                              \
    cudaError_t stencil_multi_tab_r##RR(const Job *jobs, int njobs, int total, int t, int cfg,     \
                                        cudaStream_t s, bool pdl) {                                \
        switch (cfg) {                                                                             \
            SSX_TILE_CONFIGS(SSX_CASE_MULTI_TAB)                                                   \
            default: return cudaErrorInvalidValue;                                                 \
        }                                                                                          \
    }                                                                                              \
    int stencil_capacity_r##RR(int cfg, bool adj) {                                                \
        switch (cfg) {                                                                             \
            SSX_TILE_CONFIGS(SSX_CASE_CAPACITY)                                                    \
            default: return 0;                                                                     \
        }                                                                                          \
    }                                                                                              \
    cudaError_t stencil_prepare_r##RR() {                                                          \
        cudaError_t e = cudaSuccess;                                                               \
        SSX_TILE_CONFIGS(SSX_CASE_PREPARE)                                                         \
        return e;                                                                                  \
    }

// Quads exist for order 8 only: at other orders a quad configuration runs the
// strip instance of its shape.
#define SSX_QV(V) (SSX_R == 4 ? (V) : 0)
#define SSX_CASE_FWD_STEP(id, TX, TZ, NT, V) case id: return Stencil<SSX_R>::fwd_step<TX, TZ, NT, SSX_QV(V)>(a, s, pdl);
#define SSX_CASE_ADJ_STEP(id, TX, TZ, NT, V) case id: return Stencil<SSX_R>::adj_step<TX, TZ, NT, SSX_QV(V)>(a, s, pdl);
#define SSX_CASE_FWD_PERSIST(id, TX, TZ, NT, V) case id: return Stencil<SSX_R>::fwd_persist<TX, TZ, NT, SSX_QV(V)>(a, pa, s);
#define SSX_CASE_ADJ_PERSIST(id, TX, TZ, NT, V) case id: return Stencil<SSX_R>::adj_persist<TX, TZ, NT, SSX_QV(V)>(a, pa, s);
#define SSX_CASE_MULTI(id, TX, TZ, NT, V) case id: return Stencil<SSX_R>::multi<TX, TZ, NT, SSX_QV(V)>(jobs, total, t, s, pdl);
#define SSX_CASE_MULTI_TAB(id, TX, TZ, NT, V) case id: return Stencil<SSX_R>::multi_tab<TX, TZ, NT, SSX_QV(V)>(jobs, njobs, total, t, s, pdl);
#define SSX_CASE_CAPACITY(id, TX, TZ, NT, V) case id: return Stencil<SSX_R>::capacity<TX, TZ, NT, SSX_QV(V)>(adj);
#define SSX_CASE_PREPARE(id, TX, TZ, NT, V) if (e == cudaSuccess) e = Stencil<SSX_R>::prepare<TX, TZ, NT, SSX_QV(V)>();

}  // namespace ssx
