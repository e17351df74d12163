// batch.cu -- many ligands docked in one persistent launch.
//
// The paper runs several independent GA runs per ligand at once (Section
// II-A) and screens large ligand sets; here every (ligand, run) pair is one
// task, and one warp runs a whole task -- initial population, every
// generation's children and scores, the local searches and the final pick --
// with no synchronisation beyond the warp.  Warps claim tasks from a device
// counter (largest ligands first, so the tail of the launch is short), so
// ligands of uneven size share the GPU without a per-ligand launch.  A
// task's result depends only on its ligand, run index and seed: its shared-
// memory layout is that of its own ligand and its population lives in the
// warp's own global scratch, whatever else runs beside it.
#include <math.h>

#include <algorithm>
#include <chrono>
#include <numeric>
#include <string.h>
#include <vector>

#include "ga.cuh"
#include "rescore.cuh"

namespace {

struct BatchConst {
    int pop, n_ls, iters;
    long long max_evals;
    float rho, eps;
    float p_tour, p_cross, p_mut, trans_mut;
    int gstride;  // genes per output row (DOCK_MAX_TORSIONS + 7)
    int method;   // 0 = ADADELTA, 1 = Solis-Wets
    SwConst sw;
};

BatchConst batch_const(const dock_params &P) {
    BatchConst BC;
    BC.pop = P.pop_size;
    BC.n_ls = P.ls_count;
    BC.iters = P.ls_iters;
    BC.max_evals = P.max_evals;
    BC.rho = P.rho;
    BC.eps = P.eps;
    BC.p_tour = P.p_tour;
    BC.p_cross = P.p_cross;
    BC.p_mut = P.p_mut;
    BC.trans_mut = P.trans_mut;
    BC.gstride = 7 + DOCK_MAX_TORSIONS;
    BC.method = P.ls_method;
    BC.sw.rho0 = P.sw_rho0;
    BC.sw.rho_lo = P.sw_rho_lo;
    BC.sw.expand = P.sw_expand;
    BC.sw.contract = P.sw_contract;
    BC.sw.n_succ = P.sw_succ;
    BC.sw.n_fail = P.sw_fail;
    BC.sw.step_t = P.sw_step[0];
    BC.sw.step_q = P.sw_step[1];
    BC.sw.step_tau = P.sw_step[2];
    return BC;
}

// Scratch of one warp: two populations, their energies and a pop-long
// index array for the local-search picks.
struct WarpScratch {
    float *A, *B, *EA, *EB;
    int *picks;
};

__device__ WarpScratch warp_scratch(float *base, size_t floats_per_warp, int gw, int pop, int gmax) {
    float *w = base + (size_t)gw * floats_per_warp;
    WarpScratch S;
    S.A = w;
    S.B = S.A + (size_t)pop * gmax;
    S.EA = S.B + (size_t)pop * gmax;
    S.EB = S.EA + pop;
    S.picks = reinterpret_cast<int *>(S.EB + pop);
    return S;
}

// The two local searches for one warp, kept out of line: the run loop around
// them then keeps its own registers instead of spilling them.
__device__ __noinline__ float sw_chain_warp(const LigandDev &L, const GridDev &G, float *ws, const EvalLayout &Y,
                                            float *x, float e0, int iters, const SwConst &S, uint2 key, uint32_t run,
                                            uint32_t gen, uint32_t entity, long long &n) {
    const dev::Team<1> tm(threadIdx.x & 31);
    return sw_chain<1>(L, G, ws, Y, tm, x, e0, x, iters, S, key, run, gen, entity, n);
}

__device__ __noinline__ float ls_chain_warp(const LigandDev &L, const GridDev &G, float *ws, const EvalLayout &Y,
                                            float *x, int iters, float rho, float eps) {
    const dev::Team<1> tm(threadIdx.x & 31);
    return ls_chain<1>(L, G, ws, Y, tm, x, x, iters, rho, eps);
}

// One docking run by one warp: generations until the run's evaluation count
// reaches max_evals (each adds >= pop - 1).  Returns the count.  METHOD: the
// local search compiled in (0 ADADELTA, 1 Solis-Wets, inlined), or -1: the
// one P.method names, called out of line.
template <int METHOD>
__device__ long long dock_run_warp(const LigandDev &L, const GridDev &G, const GaConst &C, const BatchConst &P,
                                   float *ws, const EvalLayout &Yn, const EvalLayout &Yg, WarpScratch S, int run,
                                   float *best_geno, float *best_E) {
    const int lane = threadIdx.x & 31, Gn = L.n_genes, pop = P.pop;
    const dev::Team<1> tm(lane);
    float *gs = ws + Yn.geno;
    for (int s = 0; s < pop; ++s) {
        if (lane == 0) init_individual(C, G, (uint32_t)run, (uint32_t)s, gs);
        __syncwarp();
        for (int j = lane; j < Gn; j += 32) S.A[(size_t)s * Gn + j] = gs[j];
        const float e = dev::eval_team<1, false>(L, G, ws, Yn, tm);
        if (lane == 0) S.EA[s] = e;
        __syncwarp();
    }
    long long evals = pop;
    for (long long gen = 1; evals < P.max_evals; ++gen) {
        const uint32_t g32 = (uint32_t)gen;
        float be;
        const int bi = run_argmin(S.EA, pop, lane, be);  // elitism
        for (int j = lane; j < Gn; j += 32) S.B[j] = S.A[(size_t)bi * Gn + j];
        if (lane == 0) S.EB[0] = be;
        for (int s = 1; s < pop; ++s) {
            long long dec[5];
            make_child(C, g32, run, s, S.A, S.EA, gs, lane, dec);
            for (int j = lane; j < Gn; j += 32) S.B[(size_t)s * Gn + j] = gs[j];
            const float e = dev::eval_team<1, false>(L, G, ws, Yn, tm);
            if (lane == 0) S.EB[s] = e;
        }
        // local-search sample: partial Fisher-Yates on the warp's scratch
        // copy of 0..pop-1 (the same picks as the one-thread list form)
        for (int i = lane; i < pop; i += 32) S.picks[i] = i;
        __syncwarp();
        if (lane == 0)
            for (int k = 0; k < P.n_ls; ++k) {
                const uint32_t w = draw4(C.key, (uint32_t)run, g32, (uint32_t)k, kLsPick, 0).x;
                const int j = k + (int)uidx(w, (uint32_t)(pop - k));
                const int t = S.picks[k];
                S.picks[k] = S.picks[j];
                S.picks[j] = t;
            }
        __syncwarp();
        long long ls_evals = 0;
        for (int k = 0; k < P.n_ls && P.iters > 0; ++k) {
            const int ind = S.picks[k];
            float *x = S.B + (size_t)ind * Gn;
            float best;
            if (METHOD == 1 || (METHOD < 0 && P.method == 1)) {
                long long n = 0;
                if (METHOD == 1)
                    best = sw_chain<1>(L, G, ws, Yn, tm, x, S.EB[ind], x, P.iters, P.sw, C.key, (uint32_t)run, g32,
                                       (uint32_t)k, n);
                else
                    best = sw_chain_warp(L, G, ws, Yn, x, S.EB[ind], P.iters, P.sw, C.key, (uint32_t)run, g32,
                                         (uint32_t)k, n);
                ls_evals += n;
            } else {
                if (METHOD == 0) best = ls_chain<1>(L, G, ws, Yg, tm, x, x, P.iters, P.rho, P.eps);
                else best = ls_chain_warp(L, G, ws, Yg, x, P.iters, P.rho, P.eps);
                ls_evals += P.iters;
            }
            __syncwarp();
            if (lane == 0) S.EB[ind] = best;
            __syncwarp();
        }
        evals += (pop - 1) + ls_evals;
        float *t = S.A; S.A = S.B; S.B = t;
        t = S.EA; S.EA = S.EB; S.EB = t;
        __syncwarp();
    }
    float be;
    const int bi = run_argmin(S.EA, pop, lane, be);
    const float *g = S.A + (size_t)bi * Gn;
    const float w = g[3], x = g[4], y = g[5], z = g[6];
    const float n = __fsqrt_rn(__fadd_rn(__fadd_rn(__fadd_rn(__fmul_rn(w, w), __fmul_rn(x, x)), __fmul_rn(y, y)),
                                         __fmul_rn(z, z)));
    for (int j = lane; j < Gn; j += 32) {
        float v = g[j];
        if (j >= 3 && j < 7 && n > 0.f) v = __fdiv_rn(v, n);
        best_geno[j] = v;
    }
    if (lane == 0) *best_E = be;
    return evals;
}

struct Task {
    int lig, run, out;
    unsigned long long seed;
};

// MINB: blocks of 128 threads per SM the registers must leave room for (4:
// <= 128 registers per thread, 3: <= 168, fewer spills); see
// DOCK_OPT_BATCH_BLOCKS.
template <int METHOD, int MINB>
__global__ void __launch_bounds__(128, MINB)
lga_persistent(const LigandDev *__restrict__ ligs, GridDev G, const Task *__restrict__ tasks, int n_tasks, int *next,
               BatchConst P, float *scratch, size_t floats_per_warp, int gmax, size_t smem_per_warp,
               float *best_geno, float *best_E32, unsigned long long *evals) {
    extern __shared__ float4 smem4[];
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    const int gw = blockIdx.x * (blockDim.x >> 5) + wib;
    float *ws = reinterpret_cast<float *>(smem4) + wib * smem_per_warp;
    const WarpScratch S = warp_scratch(scratch, floats_per_warp, gw, P.pop, gmax);
    for (;;) {
        int t = 0;
        if (lane == 0) t = atomicAdd(next, 1);
        t = __shfl_sync(0xffffffffu, t, 0);
        if (t >= n_tasks) break;
        const Task T = tasks[t];
        const LigandDev &L = ligs[T.lig];
        GaConst C;
        C.pop = P.pop;
        C.nruns = 1;
        C.nt = L.n_tors;
        C.p_tour = P.p_tour;
        C.p_cross = P.p_cross;
        C.p_mut = P.p_mut;
        C.trans_mut = P.trans_mut;
        C.key = make_uint2((uint32_t)T.seed, (uint32_t)(T.seed >> 32));
        const EvalLayout Yn = eval_layout(L.n_atoms, L.n_frag, L.nb8, false, 1);
        const EvalLayout Yg = eval_layout(L.n_atoms, L.n_frag, L.nb8, true, 1);
        const long long ev = dock_run_warp<METHOD>(L, G, C, P, ws, Yn, Yg, S, T.run,
                                                   best_geno + (size_t)T.out * P.gstride, best_E32 + T.out);
        if (lane == 0) evals[T.out] = (unsigned long long)ev;
        __syncwarp();
    }
}

__global__ void batch_rescore_kernel(const LigandDev *__restrict__ ligs, GridDev G, const Task *__restrict__ tasks,
                                     int n_tasks, int gstride, const float *best_geno, double *best_E,
                                     const unsigned long long *ev, int64_t *evals) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= n_tasks) return;
    const Task T = tasks[t];
    best_E[T.out] = rescore64_one(ligs[T.lig], G, best_geno + (size_t)T.out * gstride);
    if (evals) evals[T.out] = (int64_t)ev[T.out];
}

}  // namespace

extern "C" int dock_batch(dock_ctx *ctx, const dock_grids *grids, const dock_ligand *const *ligs, int n_ligs,
                          const dock_params *params, const uint64_t *seeds, float *best_geno, float *best_E32,
                          double *best_E, int64_t *evals_used, void *stream) {
    if (!ctx) return DOCK_ERR_INVALID;
    if (!grids || !ligs || n_ligs < 0 || !best_geno || !best_E) return set_err(ctx, DOCK_ERR_INVALID, "null argument");
    if (n_ligs == 0) return DOCK_OK;
    dock_params P;
    if (params) P = *params;
    else dock_default_params(&P);
    if (P.ls_count < 0) P.ls_count = (6 * P.pop_size + 99) / 100;
    if (P.pop_size < 2 || P.pop_size > 4096 || P.nruns < 1 || P.max_evals < 0 || P.ls_count > P.pop_size ||
        P.ls_count > 256 || P.ls_iters < 0 || !(P.rho >= 0.f && P.rho < 1.f) || !(P.eps > 0.f))
        return set_err(ctx, DOCK_ERR_INVALID, "invalid dock_params");
    if (int rc0 = check_sw(ctx, P)) return rc0;
    if (P.batch_pack != 0 && P.batch_pack != 1) return set_err(ctx, DOCK_ERR_INVALID, "batch_pack must be 0 or 1");
    cudaStream_t s = (cudaStream_t)stream;
    std::vector<LigandDev> hl(n_ligs);
    std::vector<size_t> need(n_ligs);  // shared-memory floats per warp of each ligand
    for (int k = 0; k < n_ligs; ++k) {
        if (!ligs[k]) return set_err(ctx, DOCK_ERR_INVALID, "null ligand");
        int rc = check_maps(ctx, grids, ligs[k]);
        if (rc) return rc;
        hl[k] = ligs[k]->dev;
        const LigandDev &L = hl[k];
        need[k] = (size_t)std::max(eval_layout(L.n_atoms, L.n_frag, L.nb8, true, 1).total,
                                   eval_layout(L.n_atoms, L.n_frag, L.nb8, false, 1).total);
        if (need[k] * 4 > ctx->smem_optin) return set_err(ctx, DOCK_ERR_SIZE, "ligand too large for shared memory");
    }
    // tasks: every run of every ligand, largest ligands first; with packing
    // by atom count, cut into classes of at most 32, 64, 96, 128, 255 atoms
    std::vector<int> order(n_ligs);
    std::iota(order.begin(), order.end(), 0);
    std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return hl[a].n_atoms > hl[b].n_atoms; });
    const int R = P.nruns, n_tasks = n_ligs * R;
    auto size_class = [&](int k) {
        const int n = hl[k].n_atoms;
        return P.batch_pack == 0 ? 0 : n <= 32 ? 4 : n <= 64 ? 3 : n <= 96 ? 2 : n <= 128 ? 1 : 0;
    };
    struct Cls {
        int t0, n;
        size_t smem_per_warp;
    };
    std::vector<Cls> cls;
    std::vector<Task> tasks;
    tasks.reserve(n_tasks);
    for (int k : order) {
        if (cls.empty() || size_class(k) != size_class(tasks.back().lig))
            cls.push_back(Cls{(int)tasks.size(), 0, 0});
        for (int r = 0; r < R; ++r) tasks.push_back(Task{k, r, k * R + r, seeds ? seeds[k] : (unsigned long long)k});
        cls.back().n += R;
        cls.back().smem_per_warp = std::max(cls.back().smem_per_warp, need[k]);
    }
    const int gmax = 7 + DOCK_MAX_TORSIONS;
    const size_t floats_per_warp = ((2 * (size_t)P.pop_size * gmax + 3 * (size_t)P.pop_size + 63) / 64) * 64;
    // warps per block: as asked, else by shared-memory fit; blocks to fill every SM
    if (P.batch_warps != 0 && P.batch_warps != 1 && P.batch_warps != 2 && P.batch_warps != 4)
        return set_err(ctx, DOCK_ERR_INVALID, "batch_warps must be 0, 1, 2 or 4");
    const bool b3 = ctx->batch_min_blocks == 3;
    auto kern = P.ls_method == 1 ? (b3 ? lga_persistent<1, 3> : lga_persistent<1, 4>)
                                 : (b3 ? lga_persistent<0, 3> : lga_persistent<0, 4>);
    struct Launch {
        int blocks, wpb;
        size_t smem;
    };
    std::vector<Launch> ln;
    int max_warps = 0;
    for (const Cls &c : cls) {
        int wpb = P.batch_warps ? P.batch_warps : 4;
        if (P.batch_warps && c.smem_per_warp * 4 * wpb > ctx->smem_optin)
            return set_err(ctx, DOCK_ERR_SIZE, "batch_warps: the block's shared memory does not fit");
        while (wpb > 1 && c.smem_per_warp * 4 * wpb > ctx->smem_optin) wpb >>= 1;
        const size_t smem = c.smem_per_warp * 4 * wpb;
        if (smem > 48 * 1024) {
            cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
            if (e) return cuda_err(ctx, e, "dock_batch attributes");
        }
        int per_sm = 0;
        cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, 32 * wpb, smem);
        if (e || per_sm < 1)
            return e ? cuda_err(ctx, e, "dock_batch occupancy") : set_err(ctx, DOCK_ERR_SIZE, "no occupancy");
        const int blocks = std::min(per_sm * ctx->num_sms, (c.n + wpb - 1) / wpb);
        ln.push_back(Launch{blocks, wpb, smem});
        max_warps = std::max(max_warps, blocks * wpb);
    }
    // the attribute must allow the largest block of any class
    size_t smem_max = 0;
    for (const Launch &l : ln) smem_max = std::max(smem_max, l.smem);
    if (smem_max > 48 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_max);
        if (e) return cuda_err(ctx, e, "dock_batch attributes");
    }
    const int n_cls = (int)cls.size();

    const BatchConst BC = batch_const(P);

    LigandDev *d_ligs = (LigandDev *)dev_alloc(ctx, sizeof(LigandDev) * n_ligs, s);
    Task *d_tasks = (Task *)dev_alloc(ctx, sizeof(Task) * n_tasks, s);
    int *d_next = (int *)dev_alloc(ctx, sizeof(int) * n_cls, s);
    float *scratch = (float *)dev_alloc(ctx, floats_per_warp * 4 * max_warps, s);
    unsigned long long *d_ev = (unsigned long long *)dev_alloc(ctx, 8 * (size_t)n_tasks, s);
    float *bE32 = best_E32 ? best_E32 : (float *)dev_alloc(ctx, 4 * (size_t)n_tasks, s);
    int rc = DOCK_OK;
    cudaError_t e = cudaSuccess;
    if (!d_ligs || !d_tasks || !d_next || !scratch || !d_ev || !bE32) {
        rc = set_err(ctx, DOCK_ERR_OOM, "device allocation failed in dock_batch");
    } else {
        e = cudaMemcpyAsync(d_ligs, hl.data(), sizeof(LigandDev) * n_ligs, cudaMemcpyHostToDevice, s);
        if (!e) e = cudaMemcpyAsync(d_tasks, tasks.data(), sizeof(Task) * n_tasks, cudaMemcpyHostToDevice, s);
        if (!e) e = cudaMemsetAsync(d_next, 0, sizeof(int) * n_cls, s);
        for (int c = 0; c < n_cls && !e; ++c) {
            const Launch &l = ln[c];
            TimedLaunch tl;
            timing_begin(ctx, kernel_id(ctx, "dock_batch"), s, &tl);
            kern<<<l.blocks, 32 * l.wpb, l.smem, s>>>(d_ligs, grids->dev, d_tasks + cls[c].t0, cls[c].n, d_next + c,
                                                      BC, scratch, floats_per_warp, gmax, cls[c].smem_per_warp,
                                                      best_geno, bE32, d_ev);
            timing_end(ctx, s, &tl);
            ++ctx->launches;
            e = cudaGetLastError();
        }
        if (!e) {
            batch_rescore_kernel<<<(n_tasks + 63) / 64, 64, 0, s>>>(d_ligs, grids->dev, d_tasks, n_tasks, gmax,
                                                                    best_geno, best_E, d_ev, evals_used);
            ++ctx->launches;
            e = cudaGetLastError();
        }
        // the host task list must outlive the asynchronous copy above
        if (!e) e = cudaStreamSynchronize(s);
        if (e) rc = cuda_err(ctx, e, "dock_batch kernels");
    }
    dev_free(ctx, d_ligs, s);
    dev_free(ctx, d_tasks, s);
    dev_free(ctx, d_next, s);
    dev_free(ctx, scratch, s);
    dev_free(ctx, d_ev, s);
    if (!best_E32) dev_free(ctx, bE32, s);
    return rc;
}

// ---------------------------------------------------------------------------
// Serving: the same warp-per-run docking fed from a live queue.  Requests
// become tasks in a ring that lives in mapped (zero-copy) host memory; the
// host publishes a tail count, idle warps poll it with a bounded wait and
// exit when no work arrives for a while (the host relaunches the kernel when
// new work comes).  No kernel waits on another kernel.

namespace {

struct ServeTask {
    LigandDev lig;
    GridDev grid;
    BatchConst P;
    unsigned long long seed;
    int run, out;
    int cancel;  // set by server_cancel: the warp that claims the task skips it
    int pad;
};

struct ServeCtl {
    long long tail;  // tasks published (host writes)
    int stop;        // host asks every warp to leave
    int pad;
};

// Device-side queue state. Only the warp that wins the refresh slot reads the
// host's mapped control block (at most once per kRefreshNs), so idle warps
// poll L2 instead of the host link.
struct ServeDev {
    unsigned long long head;         // next task to claim
    unsigned long long tail;         // copy of the host's published tail
    unsigned long long last_read;    // globaltimer of the last host read
    unsigned long long last_active;  // globaltimer of the last claim or completion
    unsigned long long stop;         // copy of the host's stop flag
    unsigned long long closing;      // set once the launch winds down: no warp claims any more
    unsigned long long busy;         // tasks claimed and not yet completed
};

constexpr long long kMaxPolls = 100000000;
constexpr unsigned long long kRefreshNs = 4000;

__device__ __forceinline__ unsigned long long globaltimer_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// Copies a trivially copyable struct from (mapped host) memory into shared
// memory with the warp's lanes.
template <typename T>
__device__ __forceinline__ void warp_copy(T *dst, const volatile T *src, int lane) {
    static_assert(sizeof(T) % 4 == 0, "word copy");
    const volatile uint32_t *s = reinterpret_cast<const volatile uint32_t *>(src);
    uint32_t *d = reinterpret_cast<uint32_t *>(dst);
    for (int i = lane; i < (int)(sizeof(T) / 4); i += 32) d[i] = s[i];
}

template <int MINB>
__global__ void __launch_bounds__(128, MINB)
lga_serve(const volatile ServeTask *tasks, const volatile ServeCtl *ctl, int capacity, ServeDev *q,
          float *scratch, size_t floats_per_warp, int pop_max, size_t smem_per_warp, float *best_geno,
          float *best_E32, double *best_E, unsigned long long *evals, volatile long long *done,
          unsigned long long max_idle_ns) {
    extern __shared__ float4 smem4[];
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    const int gw = blockIdx.x * (blockDim.x >> 5) + wib;
    // per warp: the task's descriptors, then the evaluator's scratch
    const size_t desc_floats = (sizeof(ServeTask) + 15) / 16 * 4;
    float *base = reinterpret_cast<float *>(smem4) + wib * (smem_per_warp + desc_floats);
    ServeTask *T = reinterpret_cast<ServeTask *>(base);
    float *ws = base + desc_floats;
    for (;;) {
        long long t = -1;
        if (lane == 0) {
            volatile ServeDev *vq = q;
            const unsigned long long idle0 = globaltimer_ns();
            for (long long polls = 0;; ++polls) {
                if (vq->stop || vq->closing) break;
                const long long h = (long long)vq->head;
                if (h < (long long)vq->tail) {
                    if ((long long)atomicCAS(&q->head, (unsigned long long)h, (unsigned long long)(h + 1)) == h) {
                        atomicAdd(&q->busy, 1ull);
                        atomicMax(&q->last_active, globaltimer_ns());
                        t = h;
                        break;
                    }
                    continue;
                }
                const unsigned long long now = globaltimer_ns(), last = vq->last_read;
                if (now - last > kRefreshNs && atomicCAS(&q->last_read, last, now) == last) {
                    if (ctl->stop) atomicExch(&q->stop, 1ull);
                    atomicMax(&q->tail, (unsigned long long)ctl->tail);
                    continue;
                }
                // bounded: once no task has been in progress for max_idle_ns the
                // launch winds down -- every warp leaves, none claims again, so
                // it ends at once and the host relaunches it for new work (a
                // launch with most warps gone would otherwise keep the few
                // left alive on new tasks and never end); the poll cap bounds
                // the wait on its own
                const unsigned long long act = max(idle0, vq->last_active);
                if ((vq->busy == 0 && now > act && now - act > max_idle_ns) || polls >= kMaxPolls) {
                    atomicExch(&q->closing, 1ull);
                    break;
                }
                __nanosleep(1000);
            }
        }
        t = __shfl_sync(0xffffffffu, t, 0);
        if (t < 0) break;
        __threadfence_system();  // the task record was written before tail
        warp_copy(T, tasks + (t % capacity), lane);
        __syncwarp();
        const LigandDev &L = T->lig;
        const GridDev &G = T->grid;
        const BatchConst &P = T->P;
        GaConst C;
        C.pop = P.pop;
        C.nruns = 1;
        C.nt = L.n_tors;
        C.p_tour = P.p_tour;
        C.p_cross = P.p_cross;
        C.p_mut = P.p_mut;
        C.trans_mut = P.trans_mut;
        C.key = make_uint2((uint32_t)T->seed, (uint32_t)(T->seed >> 32));
        const EvalLayout Yn = eval_layout(L.n_atoms, L.n_frag, L.nb8, false, 1);
        const EvalLayout Yg = eval_layout(L.n_atoms, L.n_frag, L.nb8, true, 1);
        const WarpScratch S = warp_scratch(scratch, floats_per_warp, gw, pop_max, 7 + DOCK_MAX_TORSIONS);
        const int out = T->out;
        // a cancelled task is finished at once: no evaluations, energy +inf
        const bool cancelled = ((const volatile ServeTask *)(tasks + (t % capacity)))->cancel != 0;
        long long ev = 0;
        if (!cancelled)
            ev = dock_run_warp<-1>(L, G, C, P, ws, Yn, Yg, S, T->run, best_geno + (size_t)out * P.gstride,
                                   best_E32 + out);
        __syncwarp();
        if (lane == 0) {
            best_E[out] = cancelled ? __longlong_as_double(0x7ff0000000000000ll)
                                    : rescore64_one(L, G, best_geno + (size_t)out * P.gstride);
            evals[out] = (unsigned long long)ev;
            __threadfence_system();
            done[out] = t + 1;  // completion: the task's sequence number
            atomicMax(&q->last_active, globaltimer_ns());
            atomicAdd(&q->busy, ~0ull);  // - 1
        }
        __syncwarp();
    }
}

}  // namespace

struct dock_server {
    dock_ctx *ctx = nullptr;
    cudaStream_t stream = nullptr;
    int capacity = 0, max_atoms = 0, pop_max = 0, warps = 0, wpb = 0, blocks = 0;
    size_t smem_per_warp = 0, smem = 0, floats_per_warp = 0;
    void (*kernel)(const volatile ServeTask *, const volatile ServeCtl *, int, ServeDev *, float *, size_t, int,
                   size_t, float *, float *, double *, unsigned long long *, volatile long long *,
                   unsigned long long) = nullptr;  // lga_serve at the context's register cap
    ServeTask *tasks = nullptr;  // mapped host
    ServeCtl *ctl = nullptr;     // mapped host
    long long *done = nullptr;   // mapped host
    ServeTask *d_tasks = nullptr;
    ServeCtl *d_ctl = nullptr;
    long long *d_done = nullptr;
    ServeDev *q = nullptr;
    float *scratch = nullptr, *best_geno = nullptr, *best_E32 = nullptr;
    double *best_E = nullptr;
    unsigned long long *evals = nullptr;
    long long submitted = 0;
    cudaEvent_t running = nullptr;  // recorded after each launch
    bool launched = false;
    // when server_poll last asked whether the kernel still runs: polls in
    // between trust the answer (querying the launch's event hundreds of
    // thousands of times a second was measured to slow the running kernel)
    std::chrono::steady_clock::time_point last_check{};
};

extern "C" {

int server_create(dock_ctx *ctx, int capacity, int max_atoms, int pop_max, dock_server **out) {
    if (!ctx || !out) return DOCK_ERR_INVALID;
    *out = nullptr;
    if (capacity < 1 || capacity > (1 << 22) || max_atoms < 1 || max_atoms > DOCK_MAX_ATOMS || pop_max < 2 ||
        pop_max > 4096)
        return set_err(ctx, DOCK_ERR_INVALID, "server_create: capacity, max_atoms or pop_max out of range");
    dock_server *S = new dock_server();
    S->ctx = ctx;
    S->capacity = capacity;
    S->max_atoms = max_atoms;
    S->pop_max = pop_max;
    const int nb8 = (max_atoms + 7) & ~7;
    S->smem_per_warp = (size_t)eval_layout(max_atoms, DOCK_MAX_TORSIONS + 1, nb8, true, 1).total;
    const size_t desc_floats = (sizeof(ServeTask) + 15) / 16 * 4;
    const size_t per_warp_bytes = (S->smem_per_warp + desc_floats) * 4;
    S->wpb = 4;
    while (S->wpb > 1 && per_warp_bytes * S->wpb > ctx->smem_optin) S->wpb >>= 1;
    if (per_warp_bytes > ctx->smem_optin) {
        delete S;
        return set_err(ctx, DOCK_ERR_SIZE, "server_create: max_atoms too large for shared memory");
    }
    S->smem = per_warp_bytes * S->wpb;
    cudaError_t e = cudaSuccess;
    S->kernel = ctx->batch_min_blocks == 3 ? lga_serve<3> : lga_serve<4>;
    if (S->smem > 48 * 1024) e = cudaFuncSetAttribute(S->kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)S->smem);
    int per_sm = 0;
    if (!e) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, S->kernel, 32 * S->wpb, S->smem);
    if (e || per_sm < 1) {
        delete S;
        return e ? cuda_err(ctx, e, "server_create occupancy") : set_err(ctx, DOCK_ERR_SIZE, "no occupancy");
    }
    S->blocks = per_sm * ctx->num_sms;
    S->warps = S->blocks * S->wpb;
    const int gmax = 7 + DOCK_MAX_TORSIONS;
    S->floats_per_warp = ((2 * (size_t)pop_max * gmax + 3 * (size_t)pop_max + 63) / 64) * 64;
    e = cudaHostAlloc((void **)&S->tasks, sizeof(ServeTask) * capacity, cudaHostAllocMapped);
    if (!e) e = cudaHostAlloc((void **)&S->ctl, sizeof(ServeCtl), cudaHostAllocMapped);
    if (!e) e = cudaHostAlloc((void **)&S->done, sizeof(long long) * capacity, cudaHostAllocMapped);
    if (!e) e = cudaHostGetDevicePointer((void **)&S->d_tasks, S->tasks, 0);
    if (!e) e = cudaHostGetDevicePointer((void **)&S->d_ctl, S->ctl, 0);
    if (!e) e = cudaHostGetDevicePointer((void **)&S->d_done, S->done, 0);
    if (!e) e = cudaStreamCreateWithFlags(&S->stream, cudaStreamNonBlocking);
    if (!e) e = cudaEventCreateWithFlags(&S->running, cudaEventDisableTiming);
    if (e) {
        server_destroy(S);
        return cuda_err(ctx, e, "server_create host buffers");
    }
    memset(S->ctl, 0, sizeof(ServeCtl));
    memset(S->done, 0, sizeof(long long) * capacity);
    S->q = (ServeDev *)dev_alloc(ctx, sizeof(ServeDev), S->stream);
    S->scratch = (float *)dev_alloc(ctx, S->floats_per_warp * 4 * S->warps, S->stream);
    S->best_geno = (float *)dev_alloc(ctx, (size_t)capacity * gmax * 4, S->stream);
    S->best_E32 = (float *)dev_alloc(ctx, (size_t)capacity * 4, S->stream);
    S->best_E = (double *)dev_alloc(ctx, (size_t)capacity * 8, S->stream);
    S->evals = (unsigned long long *)dev_alloc(ctx, (size_t)capacity * 8, S->stream);
    if (!S->q || !S->scratch || !S->best_geno || !S->best_E32 || !S->best_E || !S->evals) {
        server_destroy(S);
        return set_err(ctx, DOCK_ERR_OOM, "server_create device buffers");
    }
    e = cudaMemsetAsync(S->q, 0, sizeof(ServeDev), S->stream);
    if (!e) e = cudaStreamSynchronize(S->stream);
    if (e) {
        server_destroy(S);
        return cuda_err(ctx, e, "server_create");
    }
    *out = S;
    return DOCK_OK;
}

// (Re)launches the persistent kernel when none is running.
static int server_kick(dock_server *S) {
    if (S->launched && cudaEventQuery(S->running) == cudaErrorNotReady) return DOCK_OK;
    cudaGetLastError();
    const unsigned long long max_idle = 1000000000ull;  // the kernel ends after a second with no task in progress
    // the previous launch (if any) has ended: stream order puts this clear
    // after it and before the new launch
    cudaError_t e0 = cudaMemsetAsync(&S->q->closing, 0, sizeof(unsigned long long), S->stream);
    if (e0) return cuda_err(S->ctx, e0, "server launch");
    S->kernel<<<S->blocks, 32 * S->wpb, S->smem, S->stream>>>(
        S->d_tasks, S->d_ctl, S->capacity, S->q, S->scratch, S->floats_per_warp, S->pop_max, S->smem_per_warp,
        S->best_geno, S->best_E32, S->best_E, S->evals, S->d_done, max_idle);
    ++S->ctx->launches;
    cudaError_t e = cudaGetLastError();
    if (!e) e = cudaEventRecord(S->running, S->stream);
    if (e) return cuda_err(S->ctx, e, "server launch");
    S->launched = true;
    return DOCK_OK;
}

int server_submit(dock_server *S, const dock_grids *grids, const dock_ligand *lig, const dock_params *params,
                  uint64_t seed, int64_t *first_task) {
    if (!S || !grids || !lig || !first_task) return S ? set_err(S->ctx, DOCK_ERR_INVALID, "null argument") : DOCK_ERR_INVALID;
    dock_ctx *ctx = S->ctx;
    dock_params P;
    if (params) P = *params;
    else dock_default_params(&P);
    if (P.ls_count < 0) P.ls_count = (6 * P.pop_size + 99) / 100;
    if (P.pop_size < 2 || P.pop_size > S->pop_max || P.nruns < 1 || P.nruns > S->capacity || P.max_evals < 0 ||
        P.ls_count > P.pop_size || P.ls_iters < 0 || !(P.rho >= 0.f && P.rho < 1.f) || !(P.eps > 0.f))
        return set_err(ctx, DOCK_ERR_INVALID, "server_submit: invalid dock_params");
    if (int rc0 = check_sw(ctx, P)) return rc0;
    if (lig->dev.n_atoms > S->max_atoms) return set_err(ctx, DOCK_ERR_SIZE, "server_submit: ligand above max_atoms");
    int rc = check_maps(ctx, grids, lig);
    if (rc) return rc;
    // room: the oldest slot reused must be done
    const long long first = S->submitted, last = first + P.nruns - 1;
    for (long long t = std::max(0LL, first - S->capacity); t <= last - S->capacity; ++t)
        if (*(volatile long long *)&S->done[t % S->capacity] != t + 1)
            return set_err(ctx, DOCK_ERR_BUSY, "server_submit: queue full");
    const BatchConst BC = batch_const(P);
    for (int r = 0; r < P.nruns; ++r) {
        const long long t = first + r;
        ServeTask &T = S->tasks[t % S->capacity];
        T.lig = lig->dev;
        T.grid = grids->dev;
        T.P = BC;
        T.seed = seed;
        T.run = r;
        T.out = (int)(t % S->capacity);
        T.cancel = 0;
    }
    S->submitted = last + 1;
    __atomic_thread_fence(__ATOMIC_SEQ_CST);
    *(volatile long long *)&S->ctl->tail = S->submitted;  // publish
    __atomic_thread_fence(__ATOMIC_SEQ_CST);
    *first_task = first;
    return server_kick(S);
}

int server_poll(dock_server *S, int64_t first_task, int nruns, int *done) {
    if (!S || !done || nruns < 1) return S ? set_err(S->ctx, DOCK_ERR_INVALID, "invalid argument") : DOCK_ERR_INVALID;
    int all = 1;
    for (int r = 0; r < nruns && all; ++r) {
        const long long t = first_task + r;
        all = *(volatile long long *)&S->done[t % S->capacity] == t + 1;
    }
    *done = all;
    if (all) return DOCK_OK;
    // keep the kernel alive while work is pending, checking at most every ms
    const auto now = std::chrono::steady_clock::now();
    if (now - S->last_check < std::chrono::milliseconds(1)) return DOCK_OK;
    S->last_check = now;
    return server_kick(S);
}

int server_cancel(dock_server *S, int64_t first_task, int nruns) {
    if (!S || nruns < 1 || first_task < 0 || first_task + nruns > S->submitted)
        return S ? set_err(S->ctx, DOCK_ERR_INVALID, "server_cancel: not a submitted task range") : DOCK_ERR_INVALID;
    for (int r = 0; r < nruns; ++r) {
        const long long t = first_task + r;
        if (t < S->submitted - S->capacity) continue;  // its slot was reused: long finished
        *(volatile int *)&S->tasks[t % S->capacity].cancel = 1;
    }
    __atomic_thread_fence(__ATOMIC_SEQ_CST);
    return DOCK_OK;
}

int server_result(dock_server *S, int64_t first_task, int nruns, int n_genes, float *best_geno, double *best_E,
                  int64_t *evals_used) {
    if (!S || nruns < 1 || n_genes < 7 || n_genes > 7 + DOCK_MAX_TORSIONS)
        return S ? set_err(S->ctx, DOCK_ERR_INVALID, "invalid argument") : DOCK_ERR_INVALID;
    const int gmax = 7 + DOCK_MAX_TORSIONS;
    std::vector<float> g((size_t)gmax);
    for (int r = 0; r < nruns; ++r) {
        const long long t = first_task + r;
        const int slot = (int)(t % S->capacity);
        if (*(volatile long long *)&S->done[slot] != t + 1) return set_err(S->ctx, DOCK_ERR_INVALID, "result not ready");
        cudaError_t e = cudaSuccess;
        if (best_geno) {
            e = cudaMemcpy(g.data(), S->best_geno + (size_t)slot * gmax, gmax * 4, cudaMemcpyDeviceToHost);
            memcpy(best_geno + (size_t)r * n_genes, g.data(), n_genes * 4);
        }
        if (!e && best_E) e = cudaMemcpy(best_E + r, S->best_E + slot, 8, cudaMemcpyDeviceToHost);
        if (!e && evals_used) {
            unsigned long long v = 0;
            e = cudaMemcpy(&v, S->evals + slot, 8, cudaMemcpyDeviceToHost);
            evals_used[r] = (int64_t)v;
        }
        if (e) return cuda_err(S->ctx, e, "server_result");
    }
    return DOCK_OK;
}

int server_destroy(dock_server *S) {
    if (!S) return DOCK_ERR_INVALID;
    if (S->ctl) *(volatile int *)&S->ctl->stop = 1;
    __atomic_thread_fence(__ATOMIC_SEQ_CST);
    if (S->stream) cudaStreamSynchronize(S->stream);  // idle warps see stop within a refresh
    dock_ctx *ctx = S->ctx;
    dev_free(ctx, S->q, S->stream);
    dev_free(ctx, S->scratch, S->stream);
    dev_free(ctx, S->best_geno, S->stream);
    dev_free(ctx, S->best_E32, S->stream);
    dev_free(ctx, S->best_E, S->stream);
    dev_free(ctx, S->evals, S->stream);
    if (S->stream) cudaStreamSynchronize(S->stream);
    if (S->tasks) cudaFreeHost(S->tasks);
    if (S->ctl) cudaFreeHost(S->ctl);
    if (S->done) cudaFreeHost(S->done);
    if (S->running) cudaEventDestroy(S->running);
    if (S->stream) cudaStreamDestroy(S->stream);
    delete S;
    return DOCK_OK;
}

}  // extern "C"

// Device time of dock_batch at warps-per-block `wpb` (autotuning): reps
// calls after one untimed call, outputs into scratch.
int tune_batch_launch(dock_ctx *ctx, const dock_grids *grids, const dock_ligand *const *ligs, int n_ligs,
                      const dock_params &P0, int wpb, int min_blocks, int reps, double *ms) {
    dock_params P = P0;
    if (wpb) P.batch_warps = wpb;
    const int keep = ctx->batch_min_blocks;
    if (min_blocks) ctx->batch_min_blocks = min_blocks;
    const size_t rows = (size_t)n_ligs * P.nruns;
    const int gmax = 7 + DOCK_MAX_TORSIONS;
    cudaStream_t s = nullptr;
    float *g = (float *)dev_alloc(ctx, rows * gmax * 4, s);
    double *E = (double *)dev_alloc(ctx, rows * 8, s);
    int rc = DOCK_OK;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (!g || !E) rc = set_err(ctx, DOCK_ERR_OOM, "dock_tune: allocation failed");
    if (!rc && (cudaEventCreate(&e0) || cudaEventCreate(&e1))) rc = cuda_err(ctx, cudaGetLastError(), "dock_tune events");
    if (!rc) rc = dock_batch(ctx, grids, ligs, n_ligs, &P, nullptr, g, nullptr, E, nullptr, s);
    if (!rc) {
        cudaEventRecord(e0, s);
        for (int r = 0; r < reps && !rc; ++r) rc = dock_batch(ctx, grids, ligs, n_ligs, &P, nullptr, g, nullptr, E, nullptr, s);
        cudaEventRecord(e1, s);
        float t = 0.f;
        cudaError_t e = cudaEventSynchronize(e1);
        if (!e) e = cudaEventElapsedTime(&t, e0, e1);
        if (!rc && e) rc = cuda_err(ctx, e, "dock_tune timing");
        if (!rc) *ms = t / reps;
    }
    ctx->batch_min_blocks = keep;
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    dev_free(ctx, g, s);
    dev_free(ctx, E, s);
    return rc;
}
