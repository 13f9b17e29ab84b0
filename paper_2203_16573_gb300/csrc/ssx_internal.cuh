// ssx_internal.cuh -- device-side data layout and kernel interfaces shared by
// the CUDA translation units of libssx (not part of the public ABI).
#pragma once
#include <cuda.h>
#include <cuda_runtime.h>
#include <stdint.h>

namespace ssx {

// Field storage. A field of the padded grid (NZ x NX points) lives in a
// zero apron: GX columns left and right, GZ rows above and below, with the
// row pitch a multiple of 32 floats and the whole allocation rounded up to
// whole kernel tiles, so that a tile plus its 2k halo never reads outside the
// allocation and never needs a bounds test. The apron is never written, so it
// reads as the zero extension the difference operators assume.
constexpr int GX = 32;          // x apron (floats); keeps row starts 128-B aligned
constexpr int GZ = 8;           // z apron (rows) >= 2k for k <= 4
constexpr int TILE_X_MAX = 128;
constexpr int TILE_Z_MAX = 32;
constexpr int kMaxR = 4;        // order 8

struct FieldLayout {
    int NX, NZ;        // padded grid points
    int pitch;         // floats per storage row
    int rows;          // storage rows
    size_t elems() const { return (size_t)pitch * rows; }
    size_t origin() const { return (size_t)GZ * pitch + GX; }   // offset of (k=0, i=0)
};

// An injection / sampling line: columns i0 .. i0+n-1 of the padded grid at one
// depth; pressure rows kp (weight wp0) and kp+1 (wp1), v_z half rows kv (wv0)
// and kv+1 (wv1) -- linear interpolation in z; `scale` multiplies injected
// values (1 for a line density, 1/h for a point source) and, in the adjoint
// sweep, the read-out transposed injection.
struct Line {
    int i0, n;
    int kp;
    float wp0, wp1;
    int kv;
    float wv0, wv1;
    float scale;
};

// Staggered first-derivative weights c_1..c_k of order 2k (the Taylor values;
// row k, zero-padded) and their absolute sums (CFL bound).
extern const float kWeights[5][kMaxR];
extern const double kWeightsAbsSum[5];

// Storage layout of a padded grid of NX x NZ points (apron, pitch, rows).
FieldLayout field_layout(int NX, int NZ);

// Linear-interpolation weights at fractional padded-row coordinate zeta:
// rows k and k+1 with weights w0 = 1 - f, w1 = f (f < 1e-6 taken as 0).
void row_weights(double zeta, int *k, float *w0, float *w1);

// Line struct of a line at padded-row coordinate zeta (pressure rows) over
// physical columns ix0 .. ix0+n-1 of a grid of NZ padded rows, nx physical
// columns and nsp sponge points: 0 = ok, 1 = depth outside the grid,
// 2 = columns outside the physical grid.
int line_at(double zeta, int NZ, int nx, int nsp, int ix0, int n, double scale, Line *out);

// sigma_max dt / 2 of the sponge, sigma_max = 3 v_max ln(1000) / (2 nsp h)
// (0 without a sponge): the scale the sponge tables are filled with.
double sponge_scale(double v_max, int nsp, double h, double dt);

// Per-grid constant inputs of a step.
struct GridArgs {
    int NX, NZ, pitch;
    const float *kap;       // kappa dt / h at p points (origin-offset pointer)
    const float *cpk;       // C_p = B_p kappa dt / h inside the grid, 0 outside (same layout)
    const float *sxi, *sxh; // sigma dt/2 at x = i h and (i+1/2) h, [NX]
    const float *szi, *szh; // sigma dt/2 at z = k h and (k+1/2) h, [NZ]
    float cv;               // dt / (rho h)
    float c[kMaxR];         // staggered weights c_1..c_k
    int in_x0, in_x1;       // [in_x0, in_x1) x: every sponge factor is exactly 1
    int in_z0, in_z1;       // same in z (integer and half positions)
};

struct FwdArgs {
    GridArgs g;
    const float *p_in, *vx_in, *vz_in;  // origin-offset pointers
    float *p_out, *vx_out, *vz_out;
    Line src;
    const double *hsrc;   // pressure source [nt][src.n] or null
    const double *fsrc;   // velocity source [nt][src.n] or null
    Line rec;
    double *outp;         // P p   [nt][rec.n] or null (zeroed before the sweep)
    double *outv;         // P v_z [nt][rec.n] or null
    int n;                // step index
};

struct AdjArgs {
    GridArgs g;
    const float *p_in, *vx_in, *vz_in;  // adjoint state entering reverse step n
    float *p_out, *vx_out, *vz_out;
    Line src;
    double *hbar;         // adjoint of the pressure injection [nt][src.n] or null
    double *fbar;         // adjoint of the velocity injection or null
    Line rec;
    const double *yp;     // adjoint data for P p   [nt][rec.n] or null
    const double *yv;     // adjoint data for P v_z or null
    int n;                // step index (reverse sweep: nt-1 .. 0)
};

// A whole sweep in one cooperative launch (one CTA per tile, neighbour flags).
struct PersistArgs {
    float *f[2][3];              // ping-pong field triples (origin-offset pointers)
    int nt;
    int tiles_x, tiles_z;
    unsigned *flags;             // [tiles] steps completed, zeroed before the sweep
    int *err;                    // set to 1 if a neighbour wait timed out
    unsigned long long timeout_ns;
    int stall_tile;              // test hook: this tile never publishes (-1: none)
};

// One sweep of a multi-sweep launch ("phase"): sweep j advances one time
// step in launch t when 0 <= t - offset < nt. Sweeps of a phase may be
// forward or transposed, on different grids; the CTAs of launch t are split
// over the sweeps' tiles (tile_base = first CTA of the sweep). A sweep with
// offset > 0 consumes, at its step s, gather samples another sweep of the
// same phase produced in an earlier launch (lockstep chaining).
struct Job {
    int adj;                 // 0: forward sweep, 1: transposed sweep
    int offset;              // launch index of the sweep's first step
    int nt;
    int tiles_x, tile_base, tiles;
    // tile row of sweep tile tl: (tl * tx_mul) >> (32 + tx_shift) equals
    // tl / tiles_x for 0 <= tl < 2^31 (tx_shift = ceil(log2 tiles_x),
    // tx_mul = ceil(2^(32 + tx_shift) / tiles_x) < 2^33)
    unsigned long long tx_mul;
    int tx_shift;
    FwdArgs fa;              // forward: grid, lines, gathers (field pointers unused)
    AdjArgs aa;              // transposed: grid, lines, gathers
    float *f[2][3];          // ping-pong field triples (origin-offset pointers)
};
constexpr int kMaxJobs = 4;
// A sweep of a phase run by the TMA-staged kernel (order 8): its arguments and
// the tensor maps of its storage -- p, v_x, v_z of ping-pong buffers 0 and 1
// (maps 0-1, 2-3, 4-5; boxes of the tile with halos 2k x 2k, k x 0, 0 x k)
// and kappa over the tile (map 6) or, for a transposed sweep, C_p over the p box.
struct alignas(128) TmaJob {
    CUtensorMap map[7];
    Job job;
};
// A sweep of a phase run by the marching kernel (order 8, grids far larger
// than L2): its arguments and the tensor maps of its storage, boxes of one
// block of kMarchB rows -- p of ping-pong buffers 0 and 1 over the tile with a
// 2k column halo (maps 0-1), v_x with a k halo (2-3), v_z (4-5), kappa (6)
// and C_p over the p box width (7).
constexpr int kMarchB = 8;
struct alignas(128) MarchJob {
    CUtensorMap map[8];
    Job job;
};
// The sweeps of a phase, passed by value as the kernel parameter (constant
// bank): a CTA reads its sweep's arguments without a global-memory round trip.
struct JobSet {
    Job job[kMaxJobs];
    int njobs;
};

// Tile configurations of the step kernels: (id, TX, TZ, threads per CTA,
// quads). With quads = 1 the CTA has one thread per 4-column quad of one or
// two tile rows, and its interior and sponge tiles step by 16-byte vectors (order 8; at
// other orders the configuration runs as strips, like its quads = 0 twin).
// Every configuration computes bit-identical results; the runtime picks one
// per grid and direction by timing them (autotune). TX, TZ >= 2k keeps the
// halo of a persistent sweep within the four edge neighbours.
#define SSX_TILE_CONFIGS(X) \
    X(0, 64, 16, 256, 0)    \
    X(1, 64, 16, 512, 0)    \
    X(2, 32, 32, 256, 0)    \
    X(3, 64, 32, 512, 0)    \
    X(4, 64, 32, 1024, 0)   \
    X(5, 128, 16, 512, 0)   \
    X(6, 128, 32, 1024, 0)  \
    X(7, 32, 16, 256, 0)    \
    X(8, 64, 16, 256, 1)    \
    X(9, 32, 32, 256, 1)    \
    X(10, 64, 32, 512, 1)   \
    X(11, 128, 16, 512, 1)  \
    X(12, 128, 32, 1024, 1) \
    X(13, 64, 16, 128, 1)
constexpr int kNumTileCfgs = 14;
struct TileCfg {
    int tx, tz, threads;
    int quads;   // 1: interior and sponge tiles step by quads (order 8)
};
extern const TileCfg kTileCfgs[kNumTileCfgs];
// Marching-kernel shapes: (id, tile width = threads per CTA, tile height).
#define SSX_MARCH_CONFIGS(X) \
    X(0, 64, 128)            \
    X(1, 128, 64)            \
    X(2, 128, 128)           \
    X(3, 128, 32)
constexpr int kNumMarchCfgs = 4;
extern const TileCfg kMarchCfgs[kNumMarchCfgs];
// Two-step (temporally blocked) phase kernel shapes (stencil_two.cu, order 8,
// single-sweep phases): (id, TX, TZ, threads per CTA).
#define SSX_TWO_CONFIGS(X) \
    X(0, 32, 16, 256)      \
    X(1, 32, 16, 512)      \
    X(2, 32, 32, 512)
constexpr int kNumTwoCfgs = 3;
extern const TileCfg kTwoCfgs[kNumTwoCfgs];

// Kernel launchers (stencil.cu). Return the launch's cudaError_t. `pdl` sets
// programmatic dependent launch (the step waits in-kernel for the previous one).
cudaError_t launch_fwd_step(const FwdArgs &a, int R, int cfg, cudaStream_t s, bool pdl);
cudaError_t launch_adj_step(const AdjArgs &a, int R, int cfg, cudaStream_t s, bool pdl);
cudaError_t launch_fwd_persist(const FwdArgs &a, const PersistArgs &pa, int R, int cfg,
                               cudaStream_t s);
cudaError_t launch_adj_persist(const AdjArgs &a, const PersistArgs &pa, int R, int cfg,
                               cudaStream_t s);
int persist_capacity(int R, int cfg, bool adj);   // co-resident CTAs of a persistent kernel
// launch t of a phase (total_tiles CTAs)
cudaError_t launch_multi(const JobSet &jobs, int total_tiles, int t, int R, int cfg,
                         cudaStream_t s, bool pdl);
// the same with the sweeps in a device table (any number of sweeps; batches)
cudaError_t launch_multi_tab(const Job *jobs, int njobs, int total_tiles, int t, int R, int cfg,
                             cudaStream_t s, bool pdl);
cudaError_t prepare_kernels();                     // dynamic shared-memory limits (once per device)
// The TMA-staged phase kernel (stencil_tma.cu), order 8 only. Configuration
// ids above kNumTileCfgs - 1 name it: id kNumTileCfgs + k runs tile shape k.
bool tma_shape_supported(int cfg);                 // shape cfg has a TMA-staged kernel
int tma_capacity(int cfg);                         // its co-resident CTAs (the launch's grid cap)
cudaError_t prepare_tma_kernels();
// The two-step phase kernel (stencil_two.cu): launch t of a phase of one
// sweep (jobs.njobs == 1, offset 0) advances it by steps 2t and 2t + 1 (only
// 2t when `two` is false), reading buffer t mod 2 and writing the other.
cudaError_t prepare_two_kernels();
cudaError_t launch_two(const JobSet &jobs, int total_tiles, int t, bool two, int m, cudaStream_t s,
                       bool pdl);
// stall_tile >= 0 (test hook): that tile's copies are never issued, so the
// CTA's bounded wait runs out and reports error 2
cudaError_t launch_multi_tma(const TmaJob *jobs, int njobs, int total_tiles, int t, int cfg,
                             int cap, int *err, unsigned long long timeout_ns, int stall_tile,
                             cudaStream_t s, bool pdl);
// The marching phase kernel (stencil_march.cu), order 8 only: tall tiles, one
// thread per column, marched down in blocks of kMarchB rows.
int march_capacity(int m);                         // its co-resident CTAs (the launch's grid cap)
cudaError_t prepare_march_kernels();
// stall_tile >= 0 (test hook): that tile's first copies are never issued, so
// the CTA's bounded wait runs out and reports error 2
cudaError_t launch_march(const MarchJob *jobs, int njobs, int total_tiles, int t, int m, int cap,
                         int *err, unsigned long long timeout_ns, int stall_tile, cudaStream_t s,
                         bool pdl);

// per-R instantiations (stencil_r<R>.cu)
#define SSX_DECLARE_R(RR)                                                                       \
    cudaError_t stencil_fwd_step_r##RR(const FwdArgs &, int, cudaStream_t, bool);               \
    cudaError_t stencil_adj_step_r##RR(const AdjArgs &, int, cudaStream_t, bool);               \
    cudaError_t stencil_fwd_persist_r##RR(const FwdArgs &, const PersistArgs &, int, cudaStream_t); \
    cudaError_t stencil_adj_persist_r##RR(const AdjArgs &, const PersistArgs &, int, cudaStream_t); \
    cudaError_t stencil_multi_r##RR(const JobSet &, int, int, int, cudaStream_t, bool);         \
    cudaError_t stencil_multi_tab_r##RR(const Job *, int, int, int, int, cudaStream_t, bool);   \
    int stencil_capacity_r##RR(int, bool);                                                      \
    cudaError_t stencil_prepare_r##RR();
SSX_DECLARE_R(1)
SSX_DECLARE_R(2)
SSX_DECLARE_R(3)
SSX_DECLARE_R(4)
#undef SSX_DECLARE_R
cudaError_t launch_adj_init(const AdjArgs &a, int nt, cudaStream_t s);
cudaError_t launch_fill_kappa(float *kap, const FieldLayout &L, const float *vel, int nx, int nz,
                              int nsp, int row0, double rho, double dt_over_h, cudaStream_t s);
cudaError_t launch_sponge_table(float *ti, float *th, int N, int n_phys, int nsp,
                                double smax_dt_half, cudaStream_t s);
cudaError_t launch_vmax(const float *v, int n, float *out, cudaStream_t s);
// C_p = B_p kappa dt/h over a grid's whole storage (0 outside the padded grid)
cudaError_t launch_fill_cpk(const GridArgs &a, const FieldLayout &L, float *cpk, cudaStream_t s);

// FP64 Krylov kernels (krylov.cu).
constexpr int kDotBlocks = 512;
cudaError_t launch_dot(const double *a, const double *b, size_t n, double *partials,
                       double *out, cudaStream_t s);
cudaError_t launch_pcg_alpha(double *sc, cudaStream_t s);
cudaError_t launch_pcg_update(double *h, double *r, const double *p, const double *q, size_t n,
                              double *sc, double *partials, cudaStream_t s);
cudaError_t launch_pcg_beta(double *sc, cudaStream_t s);
cudaError_t launch_xpby(double *p, const double *g, size_t n, const double *sc, cudaStream_t s);
cudaError_t launch_colscale(double *out, const double *in, const double *w, int nt, int nc,
                            cudaStream_t s);
cudaError_t launch_colscale_add(double *q, const double *in, const double *w, double alpha,
                                int nt, int nc, cudaStream_t s);

// Velocity-gradient kernels (gradient.cu).
cudaError_t launch_grad_accum(double *g, const float *mu, const float *pn1, const float *pn,
                              const GridArgs &a, cudaStream_t s);
// g / kappa~ summed over each model point's padded copies (kap: kappa dt/h,
// origin-offset storage with the given pitch)
cudaError_t launch_grad_fold(double *out, const double *g, const float *vel, const float *kap,
                             int pitch, int nx, int nz, int nsp, int NX, double scale,
                             cudaStream_t s);
cudaError_t launch_residual2(double *ybar, const double *y, const double *d, size_t n,
                             cudaStream_t s);

// Device scalar slots used by the PCG kernels.
enum { SC_GR = 0, SC_PQ, SC_ALPHA, SC_RR, SC_GRNEW, SC_BETA, SC_FLAG, SC_COUNT };

}  // namespace ssx
