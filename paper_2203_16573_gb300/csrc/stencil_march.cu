// stencil_march.cu -- the phase kernel of spatial order 8 for grids far larger
// than L2: tall tiles marched down one block of rows at a time.
//
// The tile kernels (k_multi, k_multi_tma) give each thread a few rows of one
// column of a short tile. Every tile then recomputes the 2k-1 rows of v_z
// above and below it, reloads the windows of p and v_z down each column from
// shared memory for every strip, and pays its set-up (sweep, corner, step
// variant, addresses) for a handful of points per thread: on the batched
// survey that is ~210 instructions per grid point, and the step is bound by
// instruction issue, not by DRAM.
//
// Here one thread owns one column of a TX x TZ tile (TZ = 32 to 128 rows) and
// walks down it in blocks of kMarchB = 8 rows, carrying the windows down the
// column in registers: the last 2k-1 values of p (or q = C_p pbar) for the
// D+ of v_z, and the v_z of the previous block for the D- of p. Block b
//   * computes v_z on the half rows k0-k+8b .. +7 ("v_z chunk b"), which needs
//     p on rows k0-8+8b .. k0+8b+7 ("p chunks" b and b+1),
//   * for b >= 1, computes v_x on the rows of p chunk b (k0-8+8b .. k0+8b-1)
//     with its k-column halo, into shared memory,
//   * and after one barrier updates p on those rows from v_x (shared memory)
//     and from v_z chunks b-1 and b (registers).
// So every v_z row of the tile is computed once (2k-1 extra rows per tile,
// not per strip), and only the x differences read shared memory.
//
// Operands come by TMA (2-D cp.async.bulk.tensor) in blocks of 8 rows: a ring
// of three p chunks over the tile's width plus a 2k column halo, and two
// stages of the block's v_x (k halo), v_z and kappa -- or, in the transposed
// step, C_p of the next p chunk, which each thread multiplies into its own
// column (and 16 threads into the halo columns) of that chunk, keeping its
// own pbar for the update. One mbarrier per stage counts the bytes of one
// block's copies. Each thread takes what the p update needs from the block's
// buffers (its old p, kappa) into registers before the block's barrier, so
// that right after it thread 0 can refill the block's stage and ring slot
// with the copies of the block two ahead.
//
// Every point takes the arithmetic of fwd_strip / adj_strip term for term,
// through the plain formula where its block of rows and its warp's columns
// are undamped and free of lines, and through the sponge/line formula
// otherwise (which reduces to the same bits at undamped points): results are
// identical to every other tile configuration's.
//
// Waits are bounded (%globaltimer): past the limit the CTA records error 2,
// waits (bounded) for the copies it still has in flight, and returns.
#include <cuda.h>

#include <cstdint>

#include "stencil_impl.cuh"
#include "tma_ptx.cuh"

namespace ssx {
namespace {

constexpr int kR = 4;        // spatial order 8
constexpr int kB = kMarchB;  // rows per block
constexpr int kRing = 3;     // p chunks in shared memory
constexpr int kStages = 2;   // per-block operand stages
constexpr int kW = kB + 2 * kR - 1;   // p / q window down a column

template <int TX>
struct MarchSmem {
    static constexpr int PW = TX + 4 * kR, VW = TX + 2 * kR;
    static_assert(PW <= 256, "a tensor-copy box spans at most 256 elements a dimension");
    static_assert(TX % 32 == 0, "one thread a column, whole warps");
    alignas(128) float ring[kRing][kB][PW];   // p (forward) or q = C_p pbar (transposed), x = i0-2k ..
    struct alignas(128) Stage {
        alignas(128) float vx[kB][VW];        // v_x old, x = i0-k .. i0+TX+k-1, rows of p chunk b
        alignas(128) float vz[kB][TX];        // v_z old, half rows of v_z chunk b
        alignas(128) float k[kB][PW];         // kappa [kB][TX] (forward) | C_p of p chunk b+1 (transposed)
    } st[kStages];
    float vxn[kB][VW];                        // the block's new v_x (or C_v vbar_x')
    Job job;                                  // the current tile's sweep
    alignas(8) unsigned long long bar[kStages];
};

template <int TX>
constexpr size_t march_smem_bytes() { return sizeof(MarchSmem<TX>); }

// thread 0: the copies of block b of a tile (b = -1: the prologue's p chunk 0
// and, transposed, its C_p) on stage barrier (b + 3) % 3
template <int TX>
__device__ __forceinline__ void march_issue(const MarchJob *__restrict__ mj, bool adj, int odd,
                                            int i0, int k0, int b, int nb, MarchSmem<TX> &sm,
                                            unsigned bar0) {
    constexpr int PW = TX + 4 * kR, VW = TX + 2 * kR;
    const int s = (b + kStages) % kStages;
    const unsigned bar = bar0 + 8u * (unsigned)s;
    const int x0 = GX + i0, y0 = GZ + k0;   // storage coordinates of the tile corner
    unsigned bytes = sizeof(float) * kB * PW;                        // p chunk b+1
    if (adj) bytes += sizeof(float) * kB * PW;                       // C_p of that chunk
    if (b >= 0) bytes += sizeof(float) * kB * TX;                    // v_z chunk b
    if (b >= 1) bytes += sizeof(float) * kB * (VW + (adj ? 0 : TX));  // v_x (and kappa) of p chunk b
    mbar_expect_tx(bar, bytes);
    const int pc = b + 1;   // p chunk: rows k0 + 8 (pc - 1) ..
    tma_load_2d(&sm.ring[pc % kRing][0][0], &mj->map[odd], x0 - 2 * kR, y0 + kB * (pc - 1), bar);
    if (adj) tma_load_2d(&sm.st[s].k[0][0], &mj->map[7], x0 - 2 * kR, y0 + kB * (pc - 1), bar);
    if (b >= 0) tma_load_2d(&sm.st[s].vz[0][0], &mj->map[4 + odd], x0, y0 - kR + kB * b, bar);
    if (b >= 1) {
        tma_load_2d(&sm.st[s].vx[0][0], &mj->map[2 + odd], x0 - kR, y0 + kB * (b - 1), bar);
        if (!adj) tma_load_2d(&sm.st[s].k[0][0], &mj->map[6], x0, y0 + kB * (b - 1), bar);
    }
    (void)nb;
}

// Per-thread state of one tile's march.
struct MarchThread {
    int c, i;              // column in the tile, grid column
    bool colp, colx;       // p / v_z column, v_x column inside the grid
    bool wfast;            // every column of this warp undamped (sponge factor exactly 1)
    float sxi, sxh;        // sponge profile at the column
};

// ------------------------------------------------------------- forward --
// v_z chunk b of the forward step (half rows kz = k0 - k + 8b + j); `pw` holds
// p on rows k0 - 2k + 1 + 8b + w at the thread's column.
template <int TX, bool GEN>
__device__ __forceinline__ void fwd_vz(const FwdArgs &a, const MarchThread &th, int k0, int TZ,
                                       int b, int n, const float (&cc)[kR], float cv,
                                       const float (&pw)[kW], const float (&vzo)[kB][TX],
                                       float *vz_out, float (&zwin)[2 * kB]) {
    const GridArgs &g = a.g;
    const int NZ = g.NZ, pitch = g.pitch, i = th.i;
    // the rows' difference chains interleaved (each row's own order kept)
    float dd[kB];
#pragma unroll
    for (int j = 0; j < kB; j++) dd[j] = 0.0f;
#pragma unroll
    for (int m = 1; m <= kR; m++)
#pragma unroll
        for (int j = 0; j < kB; j++) dd[j] = fmaf(cc[m - 1], pw[j + kR - 1 + m] - pw[j + kR - m], dd[j]);
#pragma unroll
    for (int j = 0; j < kB; j++) {
        const int kz = k0 - kR + kB * b + j;
        const float d = dd[j];
        const float old = vzo[j][th.c];
        const bool own = kz >= k0 && kz < k0 + TZ;
        float vz;
        bool okz = true;
        if (!GEN) {
            vz = fmaf(-cv, d, old);
        } else {
            okz = th.colp && kz >= 0 && kz < NZ - 1;
            float A, B;
            damp(th.sxi + __ldg(g.szh + min(max(kz, 0), NZ - 1)), A, B);
            const float cvz = B * cv;
            vz = fmaf(-cvz, d, A * old);
            if (a.fsrc && okz) {   // vertical load f e_z delta(z - z_s)
                const float w = row_weight(kz, a.src.kv, a.src.wv0, a.src.wv1);
                const int js = i - a.src.i0;
                if (w != 0.0f && js >= 0 && js < a.src.n)
                    vz = fmaf(cvz * (w * a.src.scale), (float)a.fsrc[(size_t)n * a.src.n + js], vz);
            }
            vz = okz ? vz : 0.0f;
        }
        if (own && okz) st_out(vz_out + kz * pitch, vz);
        if (GEN && own && a.outv && okz) {   // P v_z trace
            const float w = row_weight(kz, a.rec.kv, a.rec.wv0, a.rec.wv1);
            const int jr = i - a.rec.i0;
            if (w != 0.0f && jr >= 0 && jr < a.rec.n)
                atomicAdd(&a.outv[(size_t)n * a.rec.n + jr], (double)w * (double)vz);
        }
        zwin[kB + j] = vz;
    }
}

// v_x of p chunk b (rows k = k0 - 8 + 8b + j) at the thread's column
template <int TX, bool GEN>
__device__ __forceinline__ void fwd_vx(const FwdArgs &a, const MarchThread &th, int kp0,
                                       const float (&cc)[kR], float cv,
                                       const float (&ring)[kB][TX + 4 * kR],
                                       const float (&vxo)[kB][TX + 2 * kR], float *vx_out,
                                       float (&vxn)[kB][TX + 2 * kR], float (&pold)[kB]) {
    const GridArgs &g = a.g;
    const int NZ = g.NZ, pitch = g.pitch;
    float dd[kB];
#pragma unroll
    for (int j = 0; j < kB; j++) dd[j] = 0.0f;
#pragma unroll
    for (int m = 1; m <= kR; m++)
#pragma unroll
        for (int j = 0; j < kB; j++)
            dd[j] = fmaf(cc[m - 1], ring[j][th.c + 2 * kR + m] - ring[j][th.c + 2 * kR + 1 - m], dd[j]);
#pragma unroll
    for (int j = 0; j < kB; j++) {
        const int k = kp0 + j;
        const float d = dd[j];
        const float old = vxo[j][th.c + kR];
        float vx;
        bool okx = true;
        if (!GEN) {
            vx = fmaf(-cv, d, old);
        } else {
            okx = th.colx && k < NZ;
            float A, B;
            damp(th.sxh + __ldg(g.szi + min(k, NZ - 1)), A, B);
            vx = fmaf(-(B * cv), d, A * old);
            vx = okx ? vx : 0.0f;
        }
        if (okx) st_out(vx_out + k * pitch, vx);
        vxn[j][th.c + kR] = vx;
        pold[j] = ring[j][th.c + 2 * kR];   // p^n of the row, for its update after the barrier
    }
}

// the k-column halo of v_x (columns i0-k .. i0-1 and i0+TX .. i0+TX+k-2):
// item e = r * (2k-1) + h, spread over the threads
template <int TX, bool GEN, bool ADJ>
__device__ __forceinline__ void vx_halo(const GridArgs &g, int i0, int kp0, const float (&cc)[kR],
                                        float cv, const float (&ring)[kB][TX + 4 * kR],
                                        const float (&vxo)[kB][TX + 2 * kR],
                                        float (&vxn)[kB][TX + 2 * kR]) {
    constexpr int NH = 2 * kR - 1, NI = kB * NH, NQ = (NI + TX - 1) / TX;
    const int NX = g.NX, NZ = g.NZ;
#pragma unroll
    for (int q = 0; q < NQ; q++) {
        const int e = threadIdx.x + q * TX;
        if (NI % TX != 0 && e >= NI) continue;
        const int r = e / NH, h = e - r * NH;
        const int jj = h < kR ? h : h + TX;   // v_x column: x = i0 - k + jj
        const int k = kp0 + r, x = i0 - kR + jj;
        const float *row = &ring[r][jj + kR];
        float d = 0.0f;
#pragma unroll
        for (int m = 1; m <= kR; m++) d = fmaf(cc[m - 1], row[m] - row[1 - m], d);
        const float old = vxo[r][jj];
        float val;
        if (!GEN) {
            val = ADJ ? cv * (old + d) : fmaf(-cv, d, old);
        } else {
            const bool ok = k < NZ && x >= 0 && x < NX - 1;
            float A, B;
            damp(__ldg(g.sxh + (ok ? x : 0)) + __ldg(g.szi + (ok ? k : 0)), A, B);
            if (ADJ) val = ok ? (B * cv) * (old + d) : 0.0f;
            else val = ok ? fmaf(-(B * cv), d, A * old) : 0.0f;
        }
        vxn[r][jj] = val;
    }
}

// p on the rows of p chunk b from v_x (shared memory) and v_z chunks b-1, b
template <int TX, bool GEN>
__device__ __forceinline__ void fwd_p(const FwdArgs &a, const MarchThread &th, int kp0, int n,
                                      const float (&cc)[kR], const float (&zwin)[2 * kB],
                                      const float (&vxn)[kB][TX + 2 * kR], const float (&pold)[kB],
                                      const float (&kap)[kB], float *p_out) {
    const GridArgs &g = a.g;
    const int NZ = g.NZ, pitch = g.pitch, i = th.i;
    float dd[kB];
#pragma unroll
    for (int j = 0; j < kB; j++) dd[j] = 0.0f;
#pragma unroll
    for (int m = 1; m <= kR; m++)
#pragma unroll
        for (int j = 0; j < kB; j++) {
            dd[j] = fmaf(cc[m - 1], vxn[j][th.c + kR + m - 1] - vxn[j][th.c + kR - m], dd[j]);
            dd[j] = fmaf(cc[m - 1], zwin[j + kR + m - 1] - zwin[j + kR - m], dd[j]);
        }
#pragma unroll
    for (int j = 0; j < kB; j++) {
        const int k = kp0 + j;
        const float d = dd[j];
        const float old = pold[j];
        float cp = kap[j], val;
        bool okp = true;
        if (!GEN) {
            val = fmaf(-cp, d, old);
        } else {
            okp = th.colp && k < NZ;
            float A, B;
            damp(th.sxi + __ldg(g.szi + min(k, NZ - 1)), A, B);
            cp *= B;
            val = fmaf(-cp, d, A * old);
            if (a.hsrc && okp) {   // constitutive defect h delta(z - z_s)
                const float w = row_weight(k, a.src.kp, a.src.wp0, a.src.wp1);
                const int js = i - a.src.i0;
                if (w != 0.0f && js >= 0 && js < a.src.n)
                    val = fmaf(cp * (w * a.src.scale), (float)a.hsrc[(size_t)n * a.src.n + js], val);
            }
        }
        if (okp) st_out(p_out + k * pitch, val);
        if (GEN && a.outp && okp) {   // P p trace
            const float w = row_weight(k, a.rec.kp, a.rec.wp0, a.rec.wp1);
            const int jr = i - a.rec.i0;
            if (w != 0.0f && jr >= 0 && jr < a.rec.n)
                atomicAdd(&a.outp[(size_t)n * a.rec.n + jr], (double)w * (double)val);
        }
    }
}

// ---------------------------------------------------------- transposed --
// vbar_z chunk b of the transposed step; `qw` holds q = C_p pbar on rows
// k0 - 2k + 1 + 8b + w at the thread's column
template <int TX, bool GEN>
__device__ __forceinline__ void adj_vz(const AdjArgs &a, const MarchThread &th, int k0, int TZ,
                                       int b, int n, const float (&cc)[kR], float cv,
                                       const float (&qw)[kW], const float (&vzo)[kB][TX],
                                       float *vz_out, float (&zwin)[2 * kB]) {
    const GridArgs &g = a.g;
    const int NZ = g.NZ, pitch = g.pitch, i = th.i;
    float dd[kB];
#pragma unroll
    for (int j = 0; j < kB; j++) dd[j] = 0.0f;
#pragma unroll
    for (int m = 1; m <= kR; m++)
#pragma unroll
        for (int j = 0; j < kB; j++) dd[j] = fmaf(cc[m - 1], qw[j + kR - 1 + m] - qw[j + kR - m], dd[j]);
#pragma unroll
    for (int j = 0; j < kB; j++) {
        const int kz = k0 - kR + kB * b + j;
        const float vb = vzo[j][th.c] + dd[j];
        const bool own = kz >= k0 && kz < k0 + TZ;
        float vz, out;
        bool okz = true;
        if (!GEN) {
            vz = (1.0f * cv) * vb;
            out = vb;
        } else {
            okz = th.colp && kz >= 0 && kz < NZ - 1;
            float A, B;
            damp(th.sxi + __ldg(g.szh + min(max(kz, 0), NZ - 1)), A, B);
            vz = (B * cv) * vb;
            out = A * vb;
            if (own && a.fbar && okz) {   // transposed velocity injection read out
                const float wf = row_weight(kz, a.src.kv, a.src.wv0, a.src.wv1);
                const int js = i - a.src.i0;
                if (wf != 0.0f && js >= 0 && js < a.src.n)
                    atomicAdd(&a.fbar[(size_t)n * a.src.n + js], (double)(wf * a.src.scale) * (double)vz);
            }
            if (own && a.yv && n >= 1 && okz) {   // transposed v_z sampling of step n-1
                const float wy = row_weight(kz, a.rec.kv, a.rec.wv0, a.rec.wv1);
                const int jr = i - a.rec.i0;
                if (wy != 0.0f && jr >= 0 && jr < a.rec.n)
                    out = fmaf(wy, (float)a.yv[(size_t)(n - 1) * a.rec.n + jr], out);
            }
            vz = okz ? vz : 0.0f;
        }
        if (own && okz) st_out(vz_out + kz * pitch, out);
        zwin[kB + j] = vz;
    }
}

// vbar_x' of p chunk b; the transposed pressure injection read out there
template <int TX, bool GEN>
__device__ __forceinline__ void adj_vx(const AdjArgs &a, const MarchThread &th, int kp0, int n,
                                       const float (&cc)[kR], float cv,
                                       const float (&ring)[kB][TX + 4 * kR],
                                       const float (&vxo)[kB][TX + 2 * kR], float *vx_out,
                                       float (&vxn)[kB][TX + 2 * kR]) {
    const GridArgs &g = a.g;
    const int NZ = g.NZ, pitch = g.pitch, i = th.i;
    float dd[kB];
#pragma unroll
    for (int j = 0; j < kB; j++) dd[j] = 0.0f;
#pragma unroll
    for (int m = 1; m <= kR; m++)
#pragma unroll
        for (int j = 0; j < kB; j++)
            dd[j] = fmaf(cc[m - 1], ring[j][th.c + 2 * kR + m] - ring[j][th.c + 2 * kR + 1 - m], dd[j]);
#pragma unroll
    for (int j = 0; j < kB; j++) {
        const int k = kp0 + j;
        if (GEN && a.hbar && th.colp) {   // hbar[n] = scale sum_k w_k q
            const float w = row_weight(k, a.src.kp, a.src.wp0, a.src.wp1);
            const int jl = i - a.src.i0;
            if (w != 0.0f && jl >= 0 && jl < a.src.n)
                atomicAdd(&a.hbar[(size_t)n * a.src.n + jl],
                          (double)(w * a.src.scale) * (double)ring[j][th.c + 2 * kR]);
        }
        const float vbx = vxo[j][th.c + kR] + dd[j];
        float vx, ox;
        bool okx = true;
        if (!GEN) {
            vx = cv * vbx;
            ox = vbx;
        } else {
            okx = th.colx && k < NZ;
            float A, B;
            damp(th.sxh + __ldg(g.szi + min(k, NZ - 1)), A, B);
            vx = okx ? (B * cv) * vbx : 0.0f;
            ox = A * vbx;
        }
        if (okx) st_out(vx_out + k * pitch, ox);
        vxn[j][th.c + kR] = vx;
    }
}

// pbar <- A_p pbar + D- (C_v vbar'); `rp` the thread's own pbar of the rows
template <int TX, bool GEN>
__device__ __forceinline__ void adj_p(const AdjArgs &a, const MarchThread &th, int kp0, int n,
                                      const float (&cc)[kR], const float (&zwin)[2 * kB],
                                      const float (&vxn)[kB][TX + 2 * kR], const float (&rp)[kB],
                                      float *p_out) {
    const GridArgs &g = a.g;
    const int NZ = g.NZ, pitch = g.pitch, i = th.i;
    float dd[kB];
#pragma unroll
    for (int j = 0; j < kB; j++) dd[j] = 0.0f;
#pragma unroll
    for (int m = 1; m <= kR; m++)
#pragma unroll
        for (int j = 0; j < kB; j++) {
            dd[j] = fmaf(cc[m - 1], vxn[j][th.c + kR + m - 1] - vxn[j][th.c + kR - m], dd[j]);
            dd[j] = fmaf(cc[m - 1], zwin[j + kR + m - 1] - zwin[j + kR - m], dd[j]);
        }
#pragma unroll
    for (int j = 0; j < kB; j++) {
        const int k = kp0 + j;
        const float d = dd[j];
        float out;
        bool okp = true;
        if (!GEN) {
            out = rp[j] + d;
        } else {
            okp = th.colp && k < NZ;
            float A, B;
            damp(th.sxi + __ldg(g.szi + min(k, NZ - 1)), A, B);
            out = fmaf(A, rp[j], d);
            if (a.yp && n >= 1 && okp) {   // transposed pressure sampling of step n-1
                const float w = row_weight(k, a.rec.kp, a.rec.wp0, a.rec.wp1);
                const int jr = i - a.rec.i0;
                if (w != 0.0f && jr >= 0 && jr < a.rec.n)
                    out = fmaf(w, (float)a.yp[(size_t)(n - 1) * a.rec.n + jr], out);
            }
        }
        if (okp) st_out(p_out + k * pitch, out);
    }
}

// q = C_p pbar on one p chunk, in place: the thread's own column (its pbar
// kept in `keep`) and, for the first 4k threads, one halo column each
template <int TX>
__device__ __forceinline__ void convert_chunk(float (&ring)[kB][TX + 4 * kR],
                                              const float (&cp)[kB][TX + 4 * kR], int c, bool halo,
                                              float (&keep)[kB]) {
#pragma unroll
    for (int j = 0; j < kB; j++) {
        const float pb = ring[j][c + 2 * kR];
        keep[j] = pb;
        ring[j][c + 2 * kR] = __fmul_rn(cp[j][c + 2 * kR], pb);
    }
    if (halo && c < 4 * kR) {
        const int col = c < 2 * kR ? c : c + TX;
#pragma unroll
        for (int j = 0; j < kB; j++) ring[j][col] = __fmul_rn(cp[j][col], ring[j][col]);
    }
}

// rows [lo, hi) against the line rows kl, kl + 1
__device__ __forceinline__ bool hits(int kl, int lo, int hi) { return kl + 1 >= lo && kl < hi; }

// ----------------------------------------------------------------- tile --
// One tile's march; false if a wait ran out (err set, copies drained).
template <int TX, int TZ, bool ADJ>
__device__ __forceinline__ bool march_tile(const MarchJob *__restrict__ mj, const Job &J, int i0,
                                           int k0, int st, MarchSmem<TX> &sm, unsigned bar0,
                                           unsigned &phase, int *err,
                                           unsigned long long timeout_ns, bool stall) {
    constexpr int NB = TZ / kB;
    const GridArgs &g = ADJ ? J.aa.g : J.fa.g;
    const int odd = st & 1;
    const int n = ADJ ? J.nt - 1 - st : st;
    const int c = threadIdx.x;
    MarchThread th;
    th.c = c;
    th.i = i0 + c;
    th.colp = th.i < g.NX;
    th.colx = th.i < g.NX - 1;
    th.sxi = __ldg(g.sxi + min(th.i, g.NX - 1));
    th.sxh = __ldg(g.sxh + min(th.i, g.NX - 1));
    th.wfast = __all_sync(0xffffffffu, th.i >= g.in_x0 && th.i < g.in_x1);
    // the v_x halo columns of the tile undamped and inside the grid
    const bool xhalo_in = i0 - kR >= g.in_x0 && i0 + TX + kR <= g.in_x1;
    float cc[kR];
#pragma unroll
    for (int m = 0; m < kR; m++) cc[m] = g.c[m];
    const float cv = g.cv;
    const size_t o = (size_t)th.i;
    float *p_out = J.f[odd ^ 1][0] + o, *vx_out = J.f[odd ^ 1][1] + o, *vz_out = J.f[odd ^ 1][2] + o;

    // waits in issue order: bit s of `phase` is the parity barrier s completes
    // next (it moves on only when the wait succeeded)
    auto wait = [&](int s) -> bool {
        const bool ok = __syncthreads_and(mbar_wait(bar0 + 8u * (unsigned)s, (phase >> s) & 1u, timeout_ns)) != 0;
        if (ok) phase ^= 1u << s;
        return ok;
    };
    // after a wait ran out: bounded waits for the blocks `from` .. `to` whose
    // copies were issued and may still be in flight
    auto drain = [&](int from, int to) {
        if (threadIdx.x == 0) atomicExch(err, 2);
        for (int b = from; b <= to; b++) {
            const int s = (b + kStages) % kStages;
            mbar_wait(bar0 + 8u * (unsigned)s, (phase >> s) & 1u, timeout_ns);
            phase ^= 1u << s;
        }
    };

    if (threadIdx.x == 0 && !stall) {
        march_issue<TX>(mj, ADJ, odd, i0, k0, -1, NB, sm, bar0);
        march_issue<TX>(mj, ADJ, odd, i0, k0, 0, NB, sm, bar0);
    }
    if (!wait((kStages - 1 + kStages) % kStages)) {
        if (stall) {   // nothing was issued: nothing in flight
            if (threadIdx.x == 0) atomicExch(err, 2);
        } else {
            drain(-1, 0);
        }
        return false;
    }
    // the window of p (q) down the column: rows k0-2k+1 .. k0-1 of p chunk 0
    float pw[kW], zwin[2 * kB], rp_cur[kB], rp_next[kB], pold[kB], kap[kB];
    if (ADJ) {
        convert_chunk<TX>(sm.ring[0], sm.st[kStages - 1].k, c, false, rp_next);
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");   // before TMA refills the slot
    }
#pragma unroll
    for (int w = 0; w < 2 * kR - 1; w++) pw[w] = sm.ring[0][w + 1][c + 2 * kR];
#pragma unroll
    for (int w = 0; w < 2 * kB; w++) zwin[w] = 0.0f;
#pragma unroll
    for (int j = 0; j < kB; j++) rp_cur[j] = pold[j] = kap[j] = 0.0f;
    __syncthreads();   // the prologue's stage is free again
    if (threadIdx.x == 0) march_issue<TX>(mj, ADJ, odd, i0, k0, 1, NB, sm, bar0);

    for (int b = 0; b <= NB; b++) {
        const int s = b % kStages;
        if (!wait(s)) {
            drain(b, min(b + 1, NB));
            return false;
        }
        const int pc = (b + 1) % kRing;   // p chunk b+1: new rows of the window
        if (ADJ) {
            convert_chunk<TX>(sm.ring[pc], sm.st[s].k, c, b + 1 <= NB, rp_next);
            // the converted chunk will be refilled by TMA: order the writes first
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        }
#pragma unroll
        for (int j = 0; j < kB; j++) pw[2 * kR - 1 + j] = sm.ring[pc][j][c + 2 * kR];
        // rows of this block: v_z half rows and (b >= 1) p rows
        const int kz0 = k0 - kR + kB * b, kp0 = k0 - kB + kB * b;
        const bool zin = kz0 >= g.in_z0 && kz0 + kB <= g.in_z1;
        const bool pin = kp0 >= g.in_z0 && kp0 + kB <= g.in_z1;
        const bool zfast = th.wfast && zin &&
                           (ADJ ? !((J.aa.fbar && hits(J.aa.src.kv, kz0, kz0 + kB)) ||
                                    (J.aa.yv && n >= 1 && hits(J.aa.rec.kv, kz0, kz0 + kB)))
                                : !((J.fa.fsrc && hits(J.fa.src.kv, kz0, kz0 + kB)) ||
                                    (J.fa.outv && hits(J.fa.rec.kv, kz0, kz0 + kB))));
        if (ADJ) {
            if (zfast) adj_vz<TX, false>(J.aa, th, k0, TZ, b, n, cc, cv, pw, sm.st[s].vz, vz_out, zwin);
            else adj_vz<TX, true>(J.aa, th, k0, TZ, b, n, cc, cv, pw, sm.st[s].vz, vz_out, zwin);
        } else {
            if (zfast) fwd_vz<TX, false>(J.fa, th, k0, TZ, b, n, cc, cv, pw, sm.st[s].vz, vz_out, zwin);
            else fwd_vz<TX, true>(J.fa, th, k0, TZ, b, n, cc, cv, pw, sm.st[s].vz, vz_out, zwin);
        }
        const int rc = b % kRing;   // p chunk b: the rows whose v_x and p are updated
        bool pfast = false;
        if (b >= 1) {
            const bool xfast = th.wfast && pin && (ADJ ? !(J.aa.hbar && hits(J.aa.src.kp, kp0, kp0 + kB)) : true);
            pfast = th.wfast && pin &&
                    (ADJ ? !(J.aa.yp && n >= 1 && hits(J.aa.rec.kp, kp0, kp0 + kB))
                         : !((J.fa.hsrc && hits(J.fa.src.kp, kp0, kp0 + kB)) ||
                             (J.fa.outp && hits(J.fa.rec.kp, kp0, kp0 + kB))));
            if (ADJ) {
                if (xfast) adj_vx<TX, false>(J.aa, th, kp0, n, cc, cv, sm.ring[rc], sm.st[s].vx, vx_out, sm.vxn);
                else adj_vx<TX, true>(J.aa, th, kp0, n, cc, cv, sm.ring[rc], sm.st[s].vx, vx_out, sm.vxn);
            } else {
                if (xfast) fwd_vx<TX, false>(J.fa, th, kp0, cc, cv, sm.ring[rc], sm.st[s].vx, vx_out, sm.vxn, pold);
                else fwd_vx<TX, true>(J.fa, th, kp0, cc, cv, sm.ring[rc], sm.st[s].vx, vx_out, sm.vxn, pold);
                const float(&ks)[kB][TX] = reinterpret_cast<const float(&)[kB][TX]>(sm.st[s].k);
#pragma unroll
                for (int j = 0; j < kB; j++) kap[j] = ks[j][c];
            }
            if (xhalo_in && pin) vx_halo<TX, false, ADJ>(g, i0, kp0, cc, cv, sm.ring[rc], sm.st[s].vx, sm.vxn);
            else vx_halo<TX, true, ADJ>(g, i0, kp0, cc, cv, sm.ring[rc], sm.st[s].vx, sm.vxn);
        }
        __syncthreads();   // vxn complete; the block's stage and ring slot are read out
        // copies two blocks ahead, into this block's stage and ring slot
        if (threadIdx.x == 0 && b + 2 <= NB) march_issue<TX>(mj, ADJ, odd, i0, k0, b + 2, NB, sm, bar0);
        if (b >= 1) {
            if (ADJ) {
                if (pfast) adj_p<TX, false>(J.aa, th, kp0, n, cc, zwin, sm.vxn, rp_cur, p_out);
                else adj_p<TX, true>(J.aa, th, kp0, n, cc, zwin, sm.vxn, rp_cur, p_out);
            } else {
                if (pfast) fwd_p<TX, false>(J.fa, th, kp0, n, cc, zwin, sm.vxn, pold, kap, p_out);
                else fwd_p<TX, true>(J.fa, th, kp0, n, cc, zwin, sm.vxn, pold, kap, p_out);
            }
        }
        // slide the windows by one block
#pragma unroll
        for (int w = 0; w < 2 * kR - 1; w++) pw[w] = pw[w + kB];
#pragma unroll
        for (int w = 0; w < kB; w++) zwin[w] = zwin[w + kB];
#pragma unroll
        for (int j = 0; j < kB; j++) rp_cur[j] = rp_next[j];
    }
    __syncthreads();   // every thread is done with the tile's buffers
    return true;
}

template <int TX, int TZ>
__global__ void __launch_bounds__(TX) k_march(const MarchJob *__restrict__ jobs, int njobs, int total,
                                              int t, int *err, unsigned long long timeout_ns,
                                              int stall_tile) {
    extern __shared__ __align__(128) unsigned char ssx_march_smem[];
    MarchSmem<TX> &sm = *reinterpret_cast<MarchSmem<TX> *>(ssx_march_smem);
    griddep_launch();
    if (smem_u32(ssx_march_smem) & 127u) {   // TMA destinations must be 128-byte aligned
        if (threadIdx.x == 0) atomicExch(err, 3);
        return;
    }
    const unsigned bar0 = smem_u32(&sm.bar[0]);
    if (threadIdx.x == 0) {
        for (int s = 0; s < kStages; s++) mbar_init(bar0 + 8u * (unsigned)s, 1);
        mbar_init_fence();
    }
    __syncthreads();
    griddep_wait();   // the previous step's fields are complete
    unsigned phase = 0u;
    const int G = gridDim.x;
    int j = 0;
    int tile = next_active(jobs, njobs, total, t, blockIdx.x, G, &j);
    int cur_job = -1;
    while (tile < total) {
        if (j != cur_job) {   // the sweep's arguments into shared memory
            __syncthreads();
            const int *src = reinterpret_cast<const int *>(&jobs[j].job);
            int *dst = reinterpret_cast<int *>(&sm.job);
            for (int w = threadIdx.x; w < (int)(sizeof(Job) / sizeof(int)); w += TX) dst[w] = __ldg(src + w);
            cur_job = j;
            if (threadIdx.x < 8) prefetch_map(&jobs[j].map[threadIdx.x]);
            __syncthreads();
        }
        const Job &J = sm.job;
        const int st = t - J.offset;
        int i0, k0;
        tile_corner<TX, TZ>(J.tx_mul, J.tx_shift, J.tiles_x, tile - J.tile_base, i0, k0);
        const bool stall = tile == stall_tile;
        const bool ok = J.adj ? march_tile<TX, TZ, true>(jobs + j, J, i0, k0, st, sm, bar0, phase, err, timeout_ns, stall)
                              : march_tile<TX, TZ, false>(jobs + j, J, i0, k0, st, sm, bar0, phase, err, timeout_ns, stall);
        if (!ok) return;
        const int nxt = tile + G;
        const int jend = __ldg(&jobs[j].job.tile_base) + __ldg(&jobs[j].job.tiles);
        if (nxt < jend) tile = nxt;   // same sweep, which steps in this launch
        else tile = next_active(jobs, njobs, total, t, nxt, G, &j);
    }
}

template <int TX, int TZ>
struct MarchKernel {
    static cudaError_t prepare() {
        return cudaFuncSetAttribute(k_march<TX, TZ>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    (int)march_smem_bytes<TX>());
    }
    static int capacity() {
        int dev = 0, sms = 0, per_sm = 0;
        if (cudaGetDevice(&dev) != cudaSuccess) return 0;
        if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return 0;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_march<TX, TZ>, TX,
                                                          march_smem_bytes<TX>()) != cudaSuccess)
            return 0;
        return per_sm * sms;
    }
    static cudaError_t launch(const MarchJob *jobs, int njobs, int total, int t, int *err,
                              unsigned long long timeout_ns, int stall_tile, int cap,
                              cudaStream_t s, bool pdl) {
        if (cap <= 0) return cudaErrorInvalidValue;
        cudaLaunchConfig_t cfg = {};
        cfg.gridDim = dim3(total < cap ? total : cap);
        cfg.blockDim = dim3(TX);
        cfg.dynamicSmemBytes = march_smem_bytes<TX>();
        cfg.stream = s;
        cudaLaunchAttribute at[1];
        at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
        at[0].val.programmaticStreamSerializationAllowed = 1;
        cfg.attrs = pdl ? at : nullptr;
        cfg.numAttrs = pdl ? 1 : 0;
        return cudaLaunchKernelEx(&cfg, k_march<TX, TZ>, jobs, njobs, total, t, err, timeout_ns,
                                  stall_tile);
    }
};

}  // namespace

const TileCfg kMarchCfgs[kNumMarchCfgs] = {
#define SSX_MARCH_ROW(id, TX, TZ) {TX, TZ, TX},
    SSX_MARCH_CONFIGS(SSX_MARCH_ROW)
#undef SSX_MARCH_ROW
};

int march_capacity(int m) {
    switch (m) {
#define SSX_CASE_MARCH_CAP(id, TX, TZ) case id: return MarchKernel<TX, TZ>::capacity();
        SSX_MARCH_CONFIGS(SSX_CASE_MARCH_CAP)
#undef SSX_CASE_MARCH_CAP
    }
    return 0;
}

cudaError_t prepare_march_kernels() {
    cudaError_t e = cudaSuccess;
#define SSX_CASE_MARCH_PREP(id, TX, TZ) if (e == cudaSuccess) e = MarchKernel<TX, TZ>::prepare();
    SSX_MARCH_CONFIGS(SSX_CASE_MARCH_PREP)
#undef SSX_CASE_MARCH_PREP
    return e;
}

cudaError_t launch_march(const MarchJob *jobs, int njobs, int total_tiles, int t, int m, int cap,
                         int *err, unsigned long long timeout_ns, int stall_tile, cudaStream_t s,
                         bool pdl) {
    switch (m) {
#define SSX_CASE_MARCH_LAUNCH(id, TX, TZ) \
    case id: return MarchKernel<TX, TZ>::launch(jobs, njobs, total_tiles, t, err, timeout_ns, stall_tile, cap, s, pdl);
        SSX_MARCH_CONFIGS(SSX_CASE_MARCH_LAUNCH)
#undef SSX_CASE_MARCH_LAUNCH
    }
    return cudaErrorInvalidValue;
}

}  // namespace ssx
