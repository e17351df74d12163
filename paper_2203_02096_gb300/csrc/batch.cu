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
#include <numeric>
#include <vector>

#include "ga.cuh"
#include "rescore.cuh"

namespace {

struct BatchConst {
    int pop, n_ls, iters;
    long long ngen;
    float rho, eps;
    float p_tour, p_cross, p_mut, trans_mut;
    int gstride;  // genes per output row (DOCK_MAX_TORSIONS + 7)
};

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

// One docking run by one warp.  Returns the per-run evaluation count.
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
    for (long long gen = 1; gen <= P.ngen; ++gen) {
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
        for (int k = 0; k < P.n_ls && P.iters > 0; ++k) {
            const int ind = S.picks[k];
            float *x = S.B + (size_t)ind * Gn;
            const float best = ls_chain<1>(L, G, ws, Yg, tm, x, x, P.iters, P.rho, P.eps);
            if (lane == 0) S.EB[ind] = best;
            __syncwarp();
        }
        evals += (pop - 1) + (long long)P.n_ls * P.iters;
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

__global__ void __launch_bounds__(128, 4)
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
        const long long ev = dock_run_warp(L, G, C, P, ws, Yn, Yg, S, T.run, best_geno + (size_t)T.out * P.gstride,
                                           best_E32 + T.out);
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
    cudaStream_t s = (cudaStream_t)stream;
    size_t smem_per_warp = 0;
    std::vector<LigandDev> hl(n_ligs);
    for (int k = 0; k < n_ligs; ++k) {
        if (!ligs[k]) return set_err(ctx, DOCK_ERR_INVALID, "null ligand");
        int rc = check_maps(ctx, grids, ligs[k]);
        if (rc) return rc;
        hl[k] = ligs[k]->dev;
        const LigandDev &L = hl[k];
        const size_t need = (size_t)std::max(eval_layout(L.n_atoms, L.n_frag, L.nb8, true, 1).total,
                                             eval_layout(L.n_atoms, L.n_frag, L.nb8, false, 1).total);
        smem_per_warp = std::max(smem_per_warp, need);
    }
    if (smem_per_warp * 4 > ctx->smem_optin) return set_err(ctx, DOCK_ERR_SIZE, "ligand too large for shared memory");
    // tasks: every run of every ligand, largest ligands first
    std::vector<int> order(n_ligs);
    std::iota(order.begin(), order.end(), 0);
    std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return hl[a].n_atoms > hl[b].n_atoms; });
    const int R = P.nruns, n_tasks = n_ligs * R;
    std::vector<Task> tasks;
    tasks.reserve(n_tasks);
    for (int k : order)
        for (int r = 0; r < R; ++r) tasks.push_back(Task{k, r, k * R + r, seeds ? seeds[k] : (unsigned long long)k});
    const int gmax = 7 + DOCK_MAX_TORSIONS;
    const size_t floats_per_warp = ((2 * (size_t)P.pop_size * gmax + 3 * (size_t)P.pop_size + 63) / 64) * 64;
    // warps per block by shared-memory fit; blocks to fill every SM
    int wpb = 4;
    while (wpb > 1 && smem_per_warp * 4 * wpb > ctx->smem_optin) wpb >>= 1;
    const size_t smem = smem_per_warp * 4 * wpb;
    if (smem > 48 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(lga_persistent, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e) return cuda_err(ctx, e, "dock_batch attributes");
    }
    int per_sm = 0;
    cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, lga_persistent, 32 * wpb, smem);
    if (e || per_sm < 1) return e ? cuda_err(ctx, e, "dock_batch occupancy") : set_err(ctx, DOCK_ERR_SIZE, "no occupancy");
    int blocks = per_sm * ctx->num_sms;
    blocks = std::min(blocks, (n_tasks + wpb - 1) / wpb);
    const int warps = blocks * wpb;

    BatchConst BC;
    BC.pop = P.pop_size;
    BC.n_ls = P.ls_count;
    BC.iters = P.ls_iters;
    const long long per_gen = (long long)(P.pop_size - 1) + (long long)P.ls_count * P.ls_iters;
    BC.ngen = P.max_evals > P.pop_size ? (P.max_evals - P.pop_size + per_gen - 1) / per_gen : 0;
    BC.rho = P.rho;
    BC.eps = P.eps;
    BC.p_tour = P.p_tour;
    BC.p_cross = P.p_cross;
    BC.p_mut = P.p_mut;
    BC.trans_mut = P.trans_mut;
    BC.gstride = gmax;

    LigandDev *d_ligs = (LigandDev *)dev_alloc(ctx, sizeof(LigandDev) * n_ligs, s);
    Task *d_tasks = (Task *)dev_alloc(ctx, sizeof(Task) * n_tasks, s);
    int *d_next = (int *)dev_alloc(ctx, sizeof(int), s);
    float *scratch = (float *)dev_alloc(ctx, floats_per_warp * 4 * warps, s);
    unsigned long long *d_ev = (unsigned long long *)dev_alloc(ctx, 8 * (size_t)n_tasks, s);
    float *bE32 = best_E32 ? best_E32 : (float *)dev_alloc(ctx, 4 * (size_t)n_tasks, s);
    int rc = DOCK_OK;
    if (!d_ligs || !d_tasks || !d_next || !scratch || !d_ev || !bE32) {
        rc = set_err(ctx, DOCK_ERR_OOM, "device allocation failed in dock_batch");
    } else {
        e = cudaMemcpyAsync(d_ligs, hl.data(), sizeof(LigandDev) * n_ligs, cudaMemcpyHostToDevice, s);
        if (!e) e = cudaMemcpyAsync(d_tasks, tasks.data(), sizeof(Task) * n_tasks, cudaMemcpyHostToDevice, s);
        if (!e) e = cudaMemsetAsync(d_next, 0, sizeof(int), s);
        if (!e) {
            TimedLaunch tl;
            timing_begin(ctx, kernel_id(ctx, "dock_batch"), s, &tl);
            lga_persistent<<<blocks, 32 * wpb, smem, s>>>(d_ligs, grids->dev, d_tasks, n_tasks, d_next, BC, scratch,
                                                         floats_per_warp, gmax, smem_per_warp, best_geno, bE32, d_ev);
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
