// stencil_tma.cu -- the phase kernel of spatial order 8 with its operands
// moved by the tensor memory accelerator.
//
// The plain phase kernel (k_multi_tab) gives every tile its own CTA, and each
// CTA loads its operands, waits for them, computes, and stores: on a grid far
// larger than L2 the SMs then spend most of their time waiting for DRAM. This
// kernel keeps a fixed set of CTAs resident (as many as fit on the GPU), each
// walking the tiles of the launch with a stride of the grid size, and gives
// each CTA two stages of shared memory: while it computes tile n from one
// stage, four 2-D TMA copies (cp.async.bulk.tensor) are already filling the
// other with the operands of tile n+1 -- the p (or pbar) box with its 2k halo,
// the v_x box with its k-wide column halo, the v_z box with its row halo and
// the kappa box (in the transposed step the C_p box over the p box, which the
// step overwrites with q = C_p pbar) -- and signal an mbarrier with their byte
// count. One thread issues the copies, right after the barrier that follows
// the wait for tile n (every thread has then left tile n-1, whose stage they
// refill); the address arithmetic of the loads disappears from the other
// threads. The per-point arithmetic is that of the column-strip tiles
// (fwd_strip / adj_strip, the same functions, fed from the stage), so results
// are identical to every other tile configuration's.
//
// Every mbarrier wait is bounded (%globaltimer): past the limit the CTA
// records error 2 in the context's error flag, waits (bounded again) for the
// copies it still has in flight, and returns. A shared-memory window that is
// not 128-byte aligned (never seen) records error 3 before any copy.
#include <cuda.h>

#include <cstdint>

#include "stencil_impl.cuh"
#include "tma_ptx.cuh"

namespace ssx {
namespace {

constexpr int kR = 4;   // spatial order 8: the TMA boxes' x offsets are 16-byte aligned

// One pipeline stage: the operand boxes of one tile, laid out as TMA writes
// them (row-major, no swizzle). x offsets: p and the transposed kappa box
// start at i0 - 2k, v_x at i0 - k, v_z and the forward kappa box at i0.
template <int TX, int TZ>
struct TmaStage {
    static constexpr int PH = TZ + 4 * kR, PW = TX + 4 * kR;
    static constexpr int VXB = TX + 2 * kR, VZH = TZ + 2 * kR - 1;
    alignas(128) float p[PH][PW];      // p (forward) or pbar (transposed)
    alignas(128) float vx[TZ][VXB];    // v_x, x = i0-k .. i0+TX+k-1
    alignas(128) float vz[VZH][TX];    // v_z, rows k0-k .. k0+TZ+k-2
    alignas(128) float k[PH][PW];      // kappa: [TZ][TX] at i0 (forward); C_p over the p box, then q = C_p pbar (transposed)
    static constexpr unsigned bytes(bool adj) {
        return (unsigned)(sizeof(float) * (PH * PW + TZ * VXB + VZH * TX + (adj ? PH * PW : TZ * TX)));
    }
};

template <int TX, int TZ>
struct TmaSmem {
    TmaStage<TX, TZ> st[2];
    alignas(16) float svx[TZ][TX + 2 * kR];   // C_v v_x of the step (as in TileSmem, pitch in quads)
    alignas(16) float svz[TZ + 2 * kR - 1][TX];
    Job job;                           // the current tile's sweep
    alignas(8) unsigned long long bar[2];
};

template <int TX, int TZ>
constexpr size_t tma_smem_bytes() { return sizeof(TmaSmem<TX, TZ>); }

template <int TX, int TZ, int NT, int V>
constexpr bool tma_shape_ok() {
    return StripShape<kR, TX, TZ, NT>::ok && tma_smem_bytes<TX, TZ>() <= 232448 &&
           (V == 0 || QuadShape<kR, TX, TZ, NT>::ok);
}

// ------------------------------------------------------------- operands --
// Strip operands read from a stage (same interface as GlobalIn).
template <int TX, int TZ, int NT, bool SP>
struct TmaIn {
    // true: the stage already holds the forward step's p, and every thread
    // has waited on its barrier (the copies are visible to it)
    static constexpr bool kStaged = true;
    using St = TmaStage<TX, TZ>;
    St &st;
    const GridArgs &g;
    const int i0, k0, rs, c;
    __device__ __forceinline__ TmaIn(St &st_, const GridArgs &g_, int i0_, int k0_, int rs_, int c_)
        : st(st_), g(g_), i0(i0_), k0(k0_), rs(rs_), c(c_) {}
    __device__ __forceinline__ float own_vx(int j) const { return st.vx[rs + j][c + kR]; }
    __device__ __forceinline__ float own_vz(int j) const { return st.vz[rs + j + kR][c]; }
    __device__ __forceinline__ float own_kap(int j) const {
        return reinterpret_cast<const float(*)[TX]>(&st.k[0][0])[rs + j][c];
    }
    __device__ __forceinline__ float own_p(int j) const { return st.p[rs + j + 2 * kR][c + 2 * kR]; }
    __device__ __forceinline__ float hvx(int r, int jj) const { return st.vx[r][jj]; }
    __device__ __forceinline__ float hvz(int kk, int i) const { return st.vz[kk][i - i0]; }
    // by quads (fwd_quad / adj_quad)
    __device__ __forceinline__ float4 vx4(int r, int jj) const {
        return *reinterpret_cast<const float4 *>(&st.vx[r][jj]);
    }
    __device__ __forceinline__ float4 vz4(int kk, int c4) const {
        return *reinterpret_cast<const float4 *>(&st.vz[kk][c4]);
    }
    __device__ __forceinline__ float4 kap4(int r, int c4) const {
        return *reinterpret_cast<const float4 *>(&reinterpret_cast<const float(*)[TX]>(&st.k[0][0])[r][c4]);
    }
    __device__ __forceinline__ float4 p4(int r, int c4) const {
        return *reinterpret_cast<const float4 *>(&st.p[r + 2 * kR][c4 + 2 * kR]);
    }
    // the stage is complete (every thread waited on its barrier): nothing to
    // read ahead, nothing to wait for
    static constexpr bool kAhead = true;
    static constexpr bool lines_ready = false;   // the kernel waited before the copies
    template <bool PRE>
    __device__ __forceinline__ void prestage() {}
    __device__ __forceinline__ void wait() const {}
    // transposed step: q = C_p pbar over the box, written over C_p (which
    // the step reads nowhere else; C_p is 0 outside the grid), the per-point
    // arithmetic of stage_p. Each element is read and written by one thread
    // and pbar stays in place for the others' own values: no barrier first.
    bool q_in_k = false;
    template <bool PRE>
    __device__ __forceinline__ void stage() {
        if (!PRE) return;
        constexpr int N4 = St::PH * St::PW / 4;   // by 16-byte quads (PW is a multiple of 4)
        float4 *kq = reinterpret_cast<float4 *>(&st.k[0][0]);
        const float4 *pq = reinterpret_cast<const float4 *>(&st.p[0][0]);
#pragma unroll
        for (int q = 0; q < (N4 + NT - 1) / NT; q++) {
            const int e = threadIdx.x + q * NT;
            if (N4 % NT == 0 || e < N4) {
                float4 v = kq[e];
                const float4 pv = pq[e];
                v.x = __fmul_rn(v.x, pv.x);
                v.y = __fmul_rn(v.y, pv.y);
                v.z = __fmul_rn(v.z, pv.z);
                v.w = __fmul_rn(v.w, pv.w);
                kq[e] = v;
            }
        }
        q_in_k = true;
    }
    __device__ __forceinline__ float (&sp())[TZ + 4 * kR][TX + 4 * kR] { return q_in_k ? st.k : st.p; }
};

template <int TX, int TZ, int NT, int V>
__device__ __forceinline__ void tma_tile(const Job &J, const StepIO &io, int i0, int k0,
                                         TmaStage<TX, TZ> &st, TmaSmem<TX, TZ> &sm) {
    using Q = StripShape<kR, TX, TZ, NT>;
    constexpr bool kQuads = V == 1 && QuadShape<kR, TX, TZ, NT>::ok;
    const int c = threadIdx.x % TX, rs = (threadIdx.x / TX) * Q::L;
    if (J.adj) {
        const AdjArgs &a = J.aa;
        if (adj_lines<TZ>(a, k0, io.n)) {
            TmaIn<TX, TZ, NT, true> ti(st, a.g, i0, k0, rs, c);
            adj_strip<kR, TX, TZ, NT, true, true>(a, io, i0, k0, ti, sm);
        } else if (interior_tile<kR, TX, TZ>(a.g, i0, k0)) {
            TmaIn<TX, TZ, NT, false> ti(st, a.g, i0, k0, rs, c);
            if constexpr (kQuads) adj_quad<kR, TX, TZ, NT, false>(a, io, i0, k0, ti, sm);
            else adj_strip<kR, TX, TZ, NT, false, false>(a, io, i0, k0, ti, sm);
        } else {
            TmaIn<TX, TZ, NT, true> ti(st, a.g, i0, k0, rs, c);
            if constexpr (kQuads) adj_quad<kR, TX, TZ, NT, true>(a, io, i0, k0, ti, sm);
            else adj_strip<kR, TX, TZ, NT, true, false>(a, io, i0, k0, ti, sm);
        }
    } else {
        const FwdArgs &a = J.fa;
        if (fwd_lines<kR, TZ>(a, k0)) {
            TmaIn<TX, TZ, NT, true> ti(st, a.g, i0, k0, rs, c);
            fwd_strip<kR, TX, TZ, NT, true, true>(a, io, i0, k0, ti, sm);
        } else if (interior_tile<kR, TX, TZ>(a.g, i0, k0)) {
            TmaIn<TX, TZ, NT, false> ti(st, a.g, i0, k0, rs, c);
            if constexpr (kQuads) fwd_quad<kR, TX, TZ, NT, false>(a, io, i0, k0, ti, sm);
            else fwd_strip<kR, TX, TZ, NT, false, false>(a, io, i0, k0, ti, sm);
        } else {
            TmaIn<TX, TZ, NT, true> ti(st, a.g, i0, k0, rs, c);
            if constexpr (kQuads) fwd_quad<kR, TX, TZ, NT, true>(a, io, i0, k0, ti, sm);
            else fwd_strip<kR, TX, TZ, NT, true, false>(a, io, i0, k0, ti, sm);
        }
    }
}

// thread 0: start the four copies of `tile` (sweep j) into stage `st`
template <int TX, int TZ>
__device__ __forceinline__ void issue(const TmaJob *__restrict__ jobs, int j, int tile, int t,
                                      TmaStage<TX, TZ> &st, unsigned bar) {
    const TmaJob &J = jobs[j];
    int i0, k0;
    tile_corner<TX, TZ>(__ldg(&J.job.tx_mul), __ldg(&J.job.tx_shift), __ldg(&J.job.tiles_x),
                        tile - __ldg(&J.job.tile_base), i0, k0);
    const int odd = (t - __ldg(&J.job.offset)) & 1;   // input buffer of this step
    const bool adj = __ldg(&J.job.adj) != 0;
    mbar_expect_tx(bar, TmaStage<TX, TZ>::bytes(adj));
    const int x0 = GX + i0, y0 = GZ + k0;   // storage coordinates of the tile corner
    tma_load_2d(&st.p[0][0], &J.map[odd], x0 - 2 * kR, y0 - 2 * kR, bar);
    tma_load_2d(&st.vx[0][0], &J.map[2 + odd], x0 - kR, y0, bar);
    tma_load_2d(&st.vz[0][0], &J.map[4 + odd], x0, y0 - kR, bar);
    if (adj) tma_load_2d(&st.k[0][0], &J.map[6], x0 - 2 * kR, y0 - 2 * kR, bar);
    else tma_load_2d(&st.k[0][0], &J.map[6], x0, y0, bar);
}

template <int TX, int TZ, int NT, int V>
__global__ void __launch_bounds__(NT, (NT <= 256 ? tile_min_ctas<TX, TZ, NT>() : 1))
    k_multi_tma(const TmaJob *__restrict__ jobs, int njobs, int total, int t, int *err,
                unsigned long long timeout_ns, int stall_tile) {
    // a direct cast keeps the shared address space visible to the compiler
    // (shared-memory instructions, not generic ones); the dynamic window of a
    // kernel without static shared memory starts 128-byte aligned
    extern __shared__ __align__(128) unsigned char ssx_tma_smem[];
    TmaSmem<TX, TZ> &sm = *reinterpret_cast<TmaSmem<TX, TZ> *>(ssx_tma_smem);
    griddep_launch();
    if (smem_u32(ssx_tma_smem) & 127u) {   // TMA destinations must be 128-byte aligned
        if (threadIdx.x == 0) atomicExch(err, 3);
        return;
    }
    // shared addresses of the two stage barriers: bar(s) = bar0 + 8 s (no
    // runtime-indexed local array)
    const unsigned bar0 = smem_u32(&sm.bar[0]);
    auto bar = [bar0](int k) { return bar0 + 8u * (unsigned)k; };
    if (threadIdx.x == 0) {
        mbar_init(bar(0), 1);
        mbar_init(bar(1), 1);
        mbar_init_fence();
    }

    // The tile walk, the first sweep's arguments and its tensor maps depend
    // on nothing the previous step writes. In a launch whose CTAs have one
    // tile each (a short, latency-bound step) they are fetched before the
    // grid dependency wait, while that step finishes under programmatic
    // dependent launch; a CTA with many tiles waits first and starts its
    // first copies as soon as it can.
    const int G = gridDim.x;
    const bool one_tile = total <= G;
    if (!one_tile) {
        __syncthreads();   // barriers initialised
        griddep_wait();    // the previous step's fields are complete
    }
    int j = 0, jn = 0;
    int tile = next_active(jobs, njobs, total, t, blockIdx.x, G, &j);
    // end of sweep j's tiles: a next tile below it is in the same sweep, which
    // steps in this launch, so the search can be skipped
    int jend = tile < total ? __ldg(&jobs[j].job.tile_base) + __ldg(&jobs[j].job.tiles) : 0;
    int cur_job = -1;
    if (one_tile) {
        if (tile < total) {
            const int *src = reinterpret_cast<const int *>(&jobs[j].job);
            int *dst = reinterpret_cast<int *>(&sm.job);
            for (int w = threadIdx.x; w < (int)(sizeof(Job) / sizeof(int)); w += NT) dst[w] = __ldg(src + w);
            cur_job = j;
            if (threadIdx.x < 7) prefetch_map(&jobs[j].map[threadIdx.x]);
        }
        __syncthreads();   // barriers initialised, sweep arguments in place
        griddep_wait();    // the previous step's fields are complete
    }
    // stall_tile (test hook, normally -1): that tile's copies are never issued,
    // so its wait must run out
    if (threadIdx.x == 0 && tile < total && tile != stall_tile)
        issue<TX, TZ>(jobs, j, tile, t, sm.st[0], bar(0));
    unsigned parity = 0u;   // bit s: the phase stage s waits for next
    int s = 0;
    while (tile < total) {
        int nxt = tile + G;
        if (nxt < jend) jn = j;
        else nxt = next_active(jobs, njobs, total, t, nxt, G, &jn);
        const bool ok = mbar_wait(bar(s), (parity >> s) & 1u, timeout_ns);
        if (!__syncthreads_and(ok)) {
            if (threadIdx.x == 0) atomicExch(err, 2);
            mbar_wait(bar(s), (parity >> s) & 1u, timeout_ns);   // its copies may still be in flight
            return;
        }
        parity ^= 1u << s;
        // every thread is past the previous tile: stage s ^ 1, svx, svz and
        // the job are free (its writes to stage s ^ 1 were ordered before the
        // async proxy by each thread's fence and this barrier)
        if (threadIdx.x == 0 && nxt < total && nxt != stall_tile)
            issue<TX, TZ>(jobs, jn, nxt, t, sm.st[s ^ 1], bar(s ^ 1));
        if (j != cur_job) {   // the sweep's arguments into shared memory
            const int *src = reinterpret_cast<const int *>(&jobs[j].job);
            int *dst = reinterpret_cast<int *>(&sm.job);
            for (int w = threadIdx.x; w < (int)(sizeof(Job) / sizeof(int)); w += NT) dst[w] = __ldg(src + w);
            cur_job = j;
            __syncthreads();
        }
        const Job &J = sm.job;
        const int st = t - J.offset, tl = tile - J.tile_base;
        const int odd = st & 1;
        StepIO io;
        io.p_in = io.vx_in = io.vz_in = nullptr;   // operands come from the stage
        io.p_out = J.f[odd ^ 1][0];
        io.vx_out = J.f[odd ^ 1][1];
        io.vz_out = J.f[odd ^ 1][2];
        io.n = J.adj ? J.nt - 1 - st : st;
        int i0, k0;
        tile_corner<TX, TZ>(J.tx_mul, J.tx_shift, J.tiles_x, tl, i0, k0);
        tma_tile<TX, TZ, NT, V>(J, io, i0, k0, sm.st[s], sm);
        // the transposed step rewrote stage s (q = C_p pbar over C_p) with
        // ordinary stores; order them before the copies that will refill it
        // (issued after the next tile's barrier)
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        tile = nxt;
        if (jn != j && nxt < total) jend = __ldg(&jobs[jn].job.tile_base) + __ldg(&jobs[jn].job.tiles);
        j = jn;
        s ^= 1;
    }
}

template <int TX, int TZ, int NT, int V>
struct TmaKernel {
    static cudaError_t prepare() {
        if constexpr (!tma_shape_ok<TX, TZ, NT, V>()) return cudaSuccess;
        else
            return cudaFuncSetAttribute(k_multi_tma<TX, TZ, NT, V>,
                                        cudaFuncAttributeMaxDynamicSharedMemorySize,
                                        (int)tma_smem_bytes<TX, TZ>());
    }
    static int capacity() {
        if constexpr (!tma_shape_ok<TX, TZ, NT, V>()) return 0;
        else {
            int dev = 0, sms = 0, per_sm = 0;
            if (cudaGetDevice(&dev) != cudaSuccess) return 0;
            if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return 0;
            if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_multi_tma<TX, TZ, NT, V>, NT,
                                                              tma_smem_bytes<TX, TZ>()) != cudaSuccess)
                return 0;
            return per_sm * sms;
        }
    }
    static cudaError_t launch(const TmaJob *jobs, int njobs, int total, int t, int *err,
                              unsigned long long timeout_ns, int stall_tile, int cap,
                              cudaStream_t s, bool pdl) {
        if constexpr (!tma_shape_ok<TX, TZ, NT, V>()) return cudaErrorInvalidValue;
        else {
            if (cap <= 0) return cudaErrorInvalidValue;
            cudaLaunchConfig_t cfg = {};
            cfg.gridDim = dim3(total < cap ? total : cap);
            cfg.blockDim = dim3(NT);
            cfg.dynamicSmemBytes = tma_smem_bytes<TX, TZ>();
            cfg.stream = s;
            cudaLaunchAttribute at[1];
            at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
            at[0].val.programmaticStreamSerializationAllowed = 1;
            cfg.attrs = pdl ? at : nullptr;
            cfg.numAttrs = pdl ? 1 : 0;
            return cudaLaunchKernelEx(&cfg, k_multi_tma<TX, TZ, NT, V>, jobs, njobs, total, t, err,
                                      timeout_ns, stall_tile);
        }
    }
};

}  // namespace

bool tma_shape_supported(int cfg) {
    switch (cfg) {
#define SSX_CASE_TMA_OK(id, TX, TZ, NT, V) case id: return tma_shape_ok<TX, TZ, NT, V>();
        SSX_TILE_CONFIGS(SSX_CASE_TMA_OK)
#undef SSX_CASE_TMA_OK
    }
    return false;
}

int tma_capacity(int cfg) {
    switch (cfg) {
#define SSX_CASE_TMA_CAP(id, TX, TZ, NT, V) case id: return TmaKernel<TX, TZ, NT, V>::capacity();
        SSX_TILE_CONFIGS(SSX_CASE_TMA_CAP)
#undef SSX_CASE_TMA_CAP
    }
    return 0;
}

cudaError_t prepare_tma_kernels() {
    cudaError_t e = cudaSuccess;
#define SSX_CASE_TMA_PREP(id, TX, TZ, NT, V) if (e == cudaSuccess) e = TmaKernel<TX, TZ, NT, V>::prepare();
    SSX_TILE_CONFIGS(SSX_CASE_TMA_PREP)
#undef SSX_CASE_TMA_PREP
    return e;
}

cudaError_t launch_multi_tma(const TmaJob *jobs, int njobs, int total_tiles, int t, int cfg,
                             int cap, int *err, unsigned long long timeout_ns, int stall_tile,
                             cudaStream_t s, bool pdl) {
    switch (cfg) {
#define SSX_CASE_TMA_LAUNCH(id, TX, TZ, NT, V) \
    case id: return TmaKernel<TX, TZ, NT, V>::launch(jobs, njobs, total_tiles, t, err, timeout_ns, stall_tile, cap, s, pdl);
        SSX_TILE_CONFIGS(SSX_CASE_TMA_LAUNCH)
#undef SSX_CASE_TMA_LAUNCH
    }
    return cudaErrorInvalidValue;
}

}  // namespace ssx
