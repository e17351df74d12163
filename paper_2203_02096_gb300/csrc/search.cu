// search.cu -- the Lamarckian genetic algorithm on the device (paper,
// Section II-A): initial population, elitism + tournament selection +
// two-point crossover + mutation, local-search sampling, the local search
// (ADADELTA, or the paper's Solis-Wets) with Lamarckian write-back, per-run
// evaluation counting (the per-run sum of Listing 1, folded into the
// kernels), and the driver that runs generations until the budget is spent.
//
// Genetic operators act on FP32 genes with one IEEE round-to-nearest
// operation per step (__fadd_rn & co., never contracted), so that given the
// same energies and the same Philox stream they are reproducible exactly by
// any IEEE single-precision implementation.
#include <limits.h>
#include <math.h>

#include <cmath>

#include <algorithm>
#include <mutex>
#include <string>

#include "ga.cuh"

namespace {

template <bool EVAL>
__global__ void __launch_bounds__(128)
init_kernel(LigandDev L, GridDev G, GaConst C, float *pop_out, float *E_out, unsigned long long *evals, EvalLayout W) {
    extern __shared__ float4 smem4[];
    float *ws = reinterpret_cast<float *>(smem4) + (threadIdx.x >> 5) * W.total;
    const int lane = threadIdx.x & 31;
    const dev::Team<1> tm(lane);
    const int item = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    if (item >= C.nruns * C.pop) return;
    const int r = item / C.pop, s = item % C.pop, Gn = 7 + C.nt;
    if (lane == 0) init_individual(C, G, (uint32_t)r, (uint32_t)s, ws + W.geno);
    __syncwarp();
    float *out = pop_out + (size_t)item * Gn;
    for (int j = lane; j < Gn; j += 32) out[j] = ws[W.geno + j];
    if (EVAL) {
        const float e = dev::eval_team<1, false>(L, G, ws, W, tm);
        if (lane == 0) {
            E_out[item] = e;
            if (s == 0) atomicAdd(evals + r, (unsigned long long)C.pop);
        }
    }
}

// One warp builds one child (slot s of run r) and, with EVAL, scores it.
template <bool EVAL>
__global__ void __launch_bounds__(128)
ga_kernel(LigandDev L, GridDev G, GaConst C, uint32_t gen, const float *__restrict__ pop_old,
          const float *__restrict__ E_old, float *__restrict__ pop_new, float *__restrict__ E_new,
          long long *info, unsigned long long *evals, const int *__restrict__ active, EvalLayout W) {
    extern __shared__ float4 smem4[];
    float *ws = reinterpret_cast<float *>(smem4) + (threadIdx.x >> 5) * W.total;
    const int lane = threadIdx.x & 31;
    const dev::Team<1> tm(lane);
    const int item = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    if (item >= C.nruns * C.pop) return;
    const int r = item / C.pop, s = item % C.pop, Gn = 7 + C.nt;
    const float *old = pop_old + (size_t)r * C.pop * Gn;
    const float *Eo = E_old + (size_t)r * C.pop;
    float *child = pop_new + (size_t)item * Gn;
    float *gs = ws + W.geno;
    if (active && !active[r]) {  // run finished: carry its population over unchanged
        for (int j = lane; j < Gn; j += 32) child[j] = old[(size_t)s * Gn + j];
        if (lane == 0 && E_new) E_new[item] = Eo[s];
        return;
    }
    if (s == 0) {  // elitism: the best old individual, not re-evaluated
        float be;
        const int bi = run_argmin(Eo, C.pop, lane, be);
        for (int j = lane; j < Gn; j += 32) child[j] = old[(size_t)bi * Gn + j];
        if (lane == 0) {
            if (E_new) E_new[item] = be;
            if (evals) atomicAdd(evals + r, (unsigned long long)(C.pop - 1));
            if (info) {
                long long *o = info + (size_t)item * 5;
                o[0] = bi; o[1] = bi; o[2] = 0; o[3] = 0; o[4] = 0;
            }
        }
        return;
    }
    long long dec[5];
    make_child(C, gen, r, s, old, Eo, gs, lane, dec);
    for (int j = lane; j < Gn; j += 32) child[j] = gs[j];
    if (info && lane == 0)
        for (int k = 0; k < 5; ++k) info[(size_t)item * 5 + k] = dec[k];
    if (EVAL) {
        const float e = dev::eval_team<1, false>(L, G, ws, W, tm);
        if (lane == 0) E_new[item] = e;
    }
}

// The local-search sample of a generation: the first n_ls entries of a
// partial Fisher-Yates shuffle of 0..pop-1, kept as a list of displaced
// positions instead of a pop-sized array.
__global__ void picks_kernel(int pop, int n_ls, int nruns, uint2 key, uint32_t gen, int *picks,
                             const int *__restrict__ active) {
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= nruns || (active && !active[r])) return;
    ls_picks_one(pop, n_ls, key, (uint32_t)r, gen, picks + r * n_ls);
}

// ADADELTA local search, one team of W warps per chain (W = 1: several
// one-warp teams per block; W > 1: the block is the team).  With picks
// (inside dock): chain c is pick c % n_ls of run c / n_ls, updated in place
// in the population; without: chain c starts at x_in[c] and writes x_out[c].
// trace (x, g, E null inside dock): chain c records its iterations at
// x + c iters G, g + c iters G, E + c iters.
// Residency: W = 8 keeps 3 blocks (24 warps) per SM, W = 4 three (168
// registers: the chains of a docking are too few to fill more), W = 2 six.
template <int W>
__global__ void __launch_bounds__(W == 1 ? 128 : 32 * W, W == 8 ? 3 : W == 4 ? 3 : W == 2 ? 6 : 4)
ls_kernel(LigandDev L, GridDev G, float *x_in, float *E_pop, const int *__restrict__ picks, int pop, int n_ls,
          int nchains, int iters, float rho, float eps, float *x_out, float *E_out, unsigned long long *evals,
          EvalLayout Y, LsTrace trace) {
    extern __shared__ float4 smem4[];
    const int team_in_block = W == 1 ? (threadIdx.x >> 5) : 0;
    float *ws = reinterpret_cast<float *>(smem4) + team_in_block * Y.total;
    const dev::Team<W> tm(W == 1 ? (threadIdx.x & 31) : threadIdx.x);
    const int c = W == 1 ? blockIdx.x * (blockDim.x >> 5) + team_in_block : blockIdx.x;
    if (c >= nchains) return;  // uniform over the team
    const int Gn = L.n_genes;
    float *xi, *xo, *eo;
    int run = 0;
    if (picks) {
        run = c / n_ls;
        const int ind = __ldg(picks + c);
        xi = x_in + ((size_t)run * pop + ind) * Gn;
        xo = xi;
        eo = E_pop + (size_t)run * pop + ind;
    } else {
        xi = x_in + (size_t)c * Gn;
        xo = x_out + (size_t)c * Gn;
        eo = E_out + c;
    }
    LsTrace tr{nullptr, nullptr, nullptr};
    if (trace.x) {
        const size_t o = (size_t)c * iters;
        tr = LsTrace{trace.x + o * Gn, trace.g + o * Gn, trace.E + o};
    }
    const float best = ls_chain<W>(L, G, ws, Y, tm, xi, xo, iters, rho, eps, tr);
    if (tm.rank == 0) {
        *eo = best;
        if (evals) atomicAdd(evals + run, (unsigned long long)iters);
    }
}

// Solis-Wets local search, one team of W warps per chain, as ls_kernel.
// With picks (inside dock): chain c is pick k = c % n_ls of run c / n_ls,
// starting from the individual and its stored energy, updated in place,
// entity k of the run's generation gen in the random stream; runs with
// active[run] == 0 are skipped.  Without picks: chain c starts at x_in[c]
// (energy E0[c], or evaluated when E0 is null), entity c of (run0, gen),
// and writes x_out[c], E_out[c], evals_out[c].
template <int W>
__global__ void __launch_bounds__(W == 1 ? 128 : 32 * W, W == 8 ? 3 : W == 4 ? 4 : W == 2 ? 8 : 4)
sw_kernel(LigandDev L, GridDev G, float *x_in, float *E_pop, const int *__restrict__ picks, int pop, int n_ls,
          int nchains, int iters, SwConst S, uint2 key, uint32_t run0, uint32_t gen, const float *__restrict__ E0,
          float *x_out, float *E_out, unsigned long long *evals, long long *evals_out, const int *__restrict__ active,
          EvalLayout Y) {
    extern __shared__ float4 smem4[];
    const int team_in_block = W == 1 ? (threadIdx.x >> 5) : 0;
    float *ws = reinterpret_cast<float *>(smem4) + team_in_block * Y.total;
    const dev::Team<W> tm(W == 1 ? (threadIdx.x & 31) : threadIdx.x);
    const int c = W == 1 ? blockIdx.x * (blockDim.x >> 5) + team_in_block : blockIdx.x;
    if (c >= nchains) return;  // uniform over the team
    const int Gn = L.n_genes;
    float *xi, *xo, *eo;
    float e0;
    uint32_t run = run0, entity = (uint32_t)c;
    if (picks) {
        run = (uint32_t)(c / n_ls);
        entity = (uint32_t)(c % n_ls);
        if (active && !active[run]) return;
        const int ind = __ldg(picks + c);
        xi = x_in + ((size_t)run * pop + ind) * Gn;
        xo = xi;
        eo = E_pop + (size_t)run * pop + ind;
        e0 = *eo;
    } else {
        xi = x_in + (size_t)c * Gn;
        xo = x_out + (size_t)c * Gn;
        eo = E_out + c;
        e0 = E0 ? __ldg(E0 + c) : __int_as_float(0x7fc00000);
    }
    long long n = 0;
    const float best = sw_chain<W>(L, G, ws, Y, tm, xi, e0, xo, iters, S, key, run, gen, entity, n);
    if (tm.rank == 0) {
        *eo = best;
        if (evals) atomicAdd(evals + (picks ? run : 0), (unsigned long long)n);
        if (evals_out) evals_out[c] = n;
    }
}

// After a generation of a Solis-Wets docking: run r stays active while its
// evaluation count is below the budget; status = (active runs, least count
// among them).  One block.
__global__ void gate_kernel(const unsigned long long *__restrict__ evals, int R, long long max_evals, int *active,
                            long long *status) {
    __shared__ int cnt;
    __shared__ unsigned long long lo;
    if (threadIdx.x == 0) {
        cnt = 0;
        lo = ~0ull;
    }
    __syncthreads();
    for (int r = threadIdx.x; r < R; r += blockDim.x) {
        const unsigned long long e = evals[r];
        const int a = e < (unsigned long long)max_evals;
        active[r] = a;
        if (a) {
            atomicAdd(&cnt, 1);
            atomicMin(&lo, e);
        }
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        status[0] = cnt;
        status[1] = cnt ? (long long)lo : 0;
    }
}

// Best individual of each run, quaternion normalised (FP32, fixed order).
__global__ void final_kernel(const float *__restrict__ pop, const float *__restrict__ E, int popn, int nruns, int Gn,
                             float *best_geno, float *best_E) {
    const int lane = threadIdx.x & 31;
    const int r = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    if (r >= nruns) return;
    float be;
    const int bi = run_argmin(E + (size_t)r * popn, popn, lane, be);
    const float *g = pop + ((size_t)r * popn + bi) * Gn;
    const float w = g[3], x = g[4], y = g[5], z = g[6];
    const float n = __fsqrt_rn(__fadd_rn(__fadd_rn(__fadd_rn(__fmul_rn(w, w), __fmul_rn(x, x)), __fmul_rn(y, y)),
                                         __fmul_rn(z, z)));
    for (int j = lane; j < Gn; j += 32) {
        float v = g[j];
        if (j >= 3 && j < 7 && n > 0.f) v = __fdiv_rn(v, n);
        best_geno[(size_t)r * Gn + j] = v;
    }
    if (lane == 0 && best_E) best_E[r] = be;
}

__global__ void evals_out_kernel(const unsigned long long *ev, int n, int64_t *out) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) out[i] = (int64_t)ev[i];
}

// One ADADELTA update of every gene of B points (the step ls_chain takes
// after each evaluation), torsion genes (index >= 7) wrapped to [-pi, pi).
__global__ void adadelta_step_kernel(int n, int Gn, float rho, float eps, float *x, const float *__restrict__ g,
                                     float *eg2, float *edx2) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    float xi = x[i], a = eg2[i], b = edx2[i];
    adadelta(xi, g[i], a, b, rho, eps);
    if (i % Gn >= 7) xi = wrap_any(xi);
    x[i] = xi;
    eg2[i] = a;
    edx2[i] = b;
}

__global__ void philox_kernel(const uint32_t *ctr, int n, uint2 key, uint32_t *out) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const uint4 c = make_uint4(ctr[4 * i], ctr[4 * i + 1], ctr[4 * i + 2], ctr[4 * i + 3]);
    const uint4 o = philox(c, key);
    out[4 * i] = o.x;
    out[4 * i + 1] = o.y;
    out[4 * i + 2] = o.z;
    out[4 * i + 3] = o.w;
}

// ---------------------------------------------------------------------------
// Host side

GaConst ga_const(const dock_params &p, int nt, int nruns, uint64_t seed) {
    GaConst C;
    C.pop = p.pop_size;
    C.nruns = nruns;
    C.nt = nt;
    C.p_tour = p.p_tour;
    C.p_cross = p.p_cross;
    C.p_mut = p.p_mut;
    C.trans_mut = p.trans_mut;
    C.key = make_uint2((uint32_t)seed, (uint32_t)(seed >> 32));
    return C;
}

template <typename K>
cudaError_t launch_items(dock_ctx *ctx, K kernel, int items, int warps, size_t smem, cudaStream_t s,
                         const char *name, void **args) {
    if (items <= 0) return cudaSuccess;
    if (smem > 48 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
    }
    TimedLaunch tl;
    timing_begin(ctx, kernel_id(ctx, name), s, &tl);
    cudaError_t e = cudaLaunchKernel((const void *)kernel, dim3((items + warps - 1) / warps), dim3(warps * 32), args,
                                     smem, s);
    timing_end(ctx, s, &tl);
    ++ctx->launches;
    return e;
}

int resolve_params(dock_ctx *ctx, const dock_params *in, dock_params &p) {
    if (in) p = *in;
    else dock_default_params(&p);
    if (p.ls_count < 0) p.ls_count = (6 * p.pop_size + 99) / 100;
    if (p.ls_threads != 0 && p.ls_threads != 32 && p.ls_threads != 64 && p.ls_threads != 128 && p.ls_threads != 256)
        return set_err(ctx, DOCK_ERR_INVALID, "ls_threads must be 0, 32, 64, 128 or 256");
    if (p.pop_size < 2 || p.pop_size > (1 << 20) || p.nruns < 1 || p.max_evals < 0 || p.ls_count > p.pop_size ||
        p.ls_count > kMaxLs || p.ls_iters < 0 || !(p.rho >= 0.f && p.rho < 1.f) || !(p.eps > 0.f))
        return set_err(ctx, DOCK_ERR_INVALID, "invalid dock_params");
    // kernels index individuals (run, slot) with an int
    if ((long long)p.nruns * p.pop_size > INT_MAX)
        return set_err(ctx, DOCK_ERR_INVALID, "nruns * pop_size exceeds INT_MAX");
    return check_sw(ctx, p);
}

SwConst sw_const(const dock_params &p) {
    SwConst S;
    S.rho0 = p.sw_rho0;
    S.rho_lo = p.sw_rho_lo;
    S.expand = p.sw_expand;
    S.contract = p.sw_contract;
    S.n_succ = p.sw_succ;
    S.n_fail = p.sw_fail;
    S.step_t = p.sw_step[0];
    S.step_q = p.sw_step[1];
    S.step_tau = p.sw_step[2];
    return S;
}

// Warps per local-search chain: threads_req (32..256) when given, else
// enough to put about 16 warps on every SM while chains are few; never more
// than fit in shared memory.
int ls_team_warps(const dock_ctx *ctx, int chains, int threads_req, const LigandDev &L) {
    int w = 1;
    if (threads_req > 0) {
        w = threads_req / 32;
    } else {
        // ... and only while all chains stay resident at once (teams per SM
        // as ls_kernel's launch bounds allow: 6 two-warp, 3 four- or eight-warp)
        const long long target = 16LL * ctx->num_sms;
        auto resident = [&](int tw) { return (long long)(tw == 2 ? 6 : 3) * ctx->num_sms; };
        while (w < 8 && (long long)chains * 2 * w <= target && chains <= resident(2 * w)) w <<= 1;
    }
    w = w >= 8 ? 8 : w >= 4 ? 4 : w >= 2 ? 2 : 1;
    while (w > 1 && (size_t)eval_layout(L.n_atoms, L.n_frag, L.nb8, true, w).total * 4 > ctx->smem_optin) w >>= 1;
    return w;
}

// Launches a local-search kernel at team width W (k1..k8: its W = 1, 2, 4,
// 8 instances).  W = 1: four one-warp teams per block once the chains cover
// every SM several times, else one; W > 1: one team per block.
template <typename K1, typename K2, typename K4, typename K8>
cudaError_t launch_team(dock_ctx *ctx, int W, int chains, const EvalLayout &Y, cudaStream_t s, const char *name,
                        void **args, K1 k1, K2 k2, K4 k4, K8 k8) {
    if (chains <= 0) return cudaSuccess;
    if (W == 1) {
        const int wpb = chains >= 8 * ctx->num_sms && evaluator_smem_ok(ctx, Y, 4) ? 4 : 1;
        return launch_items(ctx, k1, chains, wpb, (size_t)Y.total * 4 * wpb, s, name, args);
    }
    const size_t smem = (size_t)Y.total * 4;
    // one team per block: launch_items with "warps per item" = W
    auto go = [&](auto kernel) {
        if (smem > 48 * 1024) {
            cudaError_t e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
            if (e != cudaSuccess) return e;
        }
        TimedLaunch tl;
        timing_begin(ctx, kernel_id(ctx, name), s, &tl);
        cudaError_t e = cudaLaunchKernel((const void *)kernel, dim3(chains), dim3(32 * W), args, smem, s);
        timing_end(ctx, s, &tl);
        ++ctx->launches;
        return e;
    };
    if (W == 2) return go(k2);
    if (W == 4) return go(k4);
    return go(k8);
}

cudaError_t launch_ls(dock_ctx *ctx, int W, int chains, const EvalLayout &Y, cudaStream_t s, const char *name,
                      void **args) {
    return launch_team(ctx, W, chains, Y, s, name, args, ls_kernel<1>, ls_kernel<2>, ls_kernel<4>, ls_kernel<8>);
}

cudaError_t launch_sw(dock_ctx *ctx, int W, int chains, const EvalLayout &Y, cudaStream_t s, const char *name,
                      void **args) {
    return launch_team(ctx, W, chains, Y, s, name, args, sw_kernel<1>, sw_kernel<2>, sw_kernel<4>, sw_kernel<8>);
}

}  // namespace

extern "C" {

int dock_async(dock_ctx *ctx, const dock_grids *grids, const dock_ligand *lig, const dock_params *params,
               uint64_t seed, float *best_geno, float *best_E32, double *best_E, int64_t *evals_used, void *stream) {
    if (!ctx || !grids || !lig || !best_geno) return ctx ? set_err(ctx, DOCK_ERR_INVALID, "null argument") : DOCK_ERR_INVALID;
    dock_params P;
    int rc = resolve_params(ctx, params, P);
    if (rc) return rc;
    if ((rc = check_maps(ctx, grids, lig))) return rc;
    cudaStream_t s = (cudaStream_t)stream;
    const LigandDev &L = lig->dev;
    const GridDev &G = grids->dev;
    const int Gn = L.n_genes, pop = P.pop_size, R = P.nruns, nls = P.ls_count;
    const EvalLayout Wn = eval_layout(L.n_atoms, L.n_frag, L.nb8, false, 1);
    const int lw = ls_team_warps(ctx, P.nruns * P.ls_count, P.ls_threads, L);
    const EvalLayout Wg = eval_layout(L.n_atoms, L.n_frag, L.nb8, true, lw);
    if (!evaluator_smem_ok(ctx, Wg, 1)) return set_err(ctx, DOCK_ERR_SIZE, "ligand too large for shared memory");
    const int gw = evaluator_smem_ok(ctx, Wn, 4) ? 4 : 1;
    const size_t items = (size_t)R * pop;
    float *popA = (float *)dev_alloc(ctx, items * Gn * 4, s), *popB = (float *)dev_alloc(ctx, items * Gn * 4, s);
    float *EA = (float *)dev_alloc(ctx, items * 4, s), *EB = (float *)dev_alloc(ctx, items * 4, s);
    int *picks = (int *)dev_alloc(ctx, (size_t)R * (nls > 0 ? nls : 1) * 4, s);
    unsigned long long *ev = (unsigned long long *)dev_alloc(ctx, (size_t)R * 8, s);
    float *bE32 = best_E32 ? best_E32 : (float *)dev_alloc(ctx, (size_t)R * 4, s);
    cudaError_t e = cudaSuccess;
    if (!popA || !popB || !EA || !EB || !picks || !ev || !bE32) {
        rc = set_err(ctx, DOCK_ERR_OOM, "device allocation failed in dock");
        goto done;
    }
    {
        GaConst C = ga_const(P, L.n_tors, R, seed);
        LigandDev l = L;
        GridDev g = G;
        EvalLayout wn = Wn, wg = Wg;
        e = cudaMemsetAsync(ev, 0, (size_t)R * 8, s);
        {
            void *a[] = {&l, &g, &C, &popA, &EA, &ev, &wn};
            if (!e) e = launch_items(ctx, init_kernel<true>, (int)items, gw, (size_t)Wn.total * 4 * gw, s, "dock_init", a);
        }
        const int chains = R * nls;
        long long *no_info = nullptr;
        float *no_out = nullptr;
        int *no_active = nullptr;
        if (P.ls_method == 0) {
            const long long per_gen = (long long)(pop - 1) + (long long)nls * P.ls_iters;
            long long ngen = 0;
            if (P.max_evals > pop) ngen = (P.max_evals - pop + per_gen - 1) / per_gen;
            for (long long gen = 1; gen <= ngen && !e; ++gen) {
                uint32_t g32 = (uint32_t)gen;
                void *a[] = {&l, &g, &C, &g32, &popA, &EA, &popB, &EB, &no_info, &ev, &no_active, &wn};
                e = launch_items(ctx, ga_kernel<true>, (int)items, gw, (size_t)Wn.total * 4 * gw, s, "dock_ga", a);
                if (!e && chains > 0 && P.ls_iters > 0) {
                    TimedLaunch tl;
                    timing_begin(ctx, kernel_id(ctx, "dock_picks"), s, &tl);
                    picks_kernel<<<(R + 63) / 64, 64, 0, s>>>(pop, nls, R, C.key, g32, picks, no_active);
                    timing_end(ctx, s, &tl);
                    ++ctx->launches;
                    e = cudaGetLastError();
                    int iters = P.ls_iters;
                    float rho = P.rho, eps = P.eps;
                    int nl = nls, ch = chains, popn = pop;
                    LsTrace no_trace{nullptr, nullptr, nullptr};
                    void *c[] = {&l,   &g,   &popB,   &EB,     &picks, &popn, &nl,      &ch,
                                 &iters, &rho, &eps, &no_out, &no_out, &ev,   &wg,  &no_trace};
                    if (!e) e = launch_ls(ctx, lw, chains, Wg, s, "dock_ls", c);
                }
                std::swap(popA, popB);
                std::swap(EA, EB);
            }
        } else if (P.max_evals > pop) {
            // Solis-Wets: a run's count per generation depends on its searches,
            // so runs are gated on the device and the host queues generations
            // in chunks, reading (active runs, least count) after each.
            const EvalLayout Ws = eval_layout(L.n_atoms, L.n_frag, L.nb8, false, lw);
            int *active = (int *)dev_alloc(ctx, (size_t)R * 4, s);
            long long *status = (long long *)dev_alloc(ctx, 16, s);
            long long *h = host_status(ctx);
            if (!active || !status || !h) {
                rc = set_err(ctx, DOCK_ERR_OOM, "allocation failed in dock (Solis-Wets state)");
            } else {
                SwConst S = sw_const(P);
                const long long per_gen_hi = (long long)(pop - 1) + 2LL * nls * P.ls_iters;
                const long long cap = P.max_evals / (pop - 1) + 2;  // each generation adds >= pop - 1
                long long gen = 0, chunk = std::max(1LL, (P.max_evals - pop) / per_gen_hi);
                const long long mx = P.max_evals;
                gate_kernel<<<1, 256, 0, s>>>(ev, R, mx, active, status);
                ++ctx->launches;
                e = cudaGetLastError();
                while (!e && gen < cap) {
                    for (long long i = 0; i < chunk && gen < cap && !e; ++i) {
                        ++gen;
                        uint32_t g32 = (uint32_t)gen;
                        void *a[] = {&l, &g, &C, &g32, &popA, &EA, &popB, &EB, &no_info, &ev, &active, &wn};
                        e = launch_items(ctx, ga_kernel<true>, (int)items, gw, (size_t)Wn.total * 4 * gw, s, "dock_ga", a);
                        if (!e && chains > 0 && P.ls_iters > 0) {
                            picks_kernel<<<(R + 63) / 64, 64, 0, s>>>(pop, nls, R, C.key, g32, picks, active);
                            ++ctx->launches;
                            e = cudaGetLastError();
                            int iters = P.ls_iters, nl = nls, ch = chains, popn = pop;
                            uint32_t run0 = 0;
                            const float *no_e0 = nullptr;
                            long long *no_eo = nullptr;
                            EvalLayout ws_ = Ws;
                            void *c[] = {&l, &g, &popB, &EB, &picks, &popn, &nl, &ch, &iters, &S, &C.key, &run0, &g32,
                                         &no_e0, &no_out, &no_out, &ev, &no_eo, &active, &ws_};
                            if (!e) e = launch_sw(ctx, lw, chains, Ws, s, "dock_sw", c);
                        }
                        if (!e) {
                            gate_kernel<<<1, 256, 0, s>>>(ev, R, mx, active, status);
                            ++ctx->launches;
                            e = cudaGetLastError();
                        }
                        std::swap(popA, popB);
                        std::swap(EA, EB);
                    }
                    if (!e) e = cudaMemcpyAsync(h, status, 16, cudaMemcpyDeviceToHost, s);
                    if (!e) e = cudaStreamSynchronize(s);
                    if (e || h[0] == 0) break;
                    // the least-advanced run's mean count per generation so far
                    const double rate = std::max(1.0, (double)(h[1] - pop) / (double)gen);
                    chunk = std::max(1LL, (long long)std::ceil((double)(P.max_evals - h[1]) / rate));
                }
            }
            dev_free(ctx, active, s);
            dev_free(ctx, status, s);
        }
        if (!e) {
            TimedLaunch tl;
            timing_begin(ctx, kernel_id(ctx, "dock_final"), s, &tl);
            final_kernel<<<(R + 3) / 4, 128, 0, s>>>(popA, EA, pop, R, Gn, best_geno, bE32);
            timing_end(ctx, s, &tl);
            ++ctx->launches;
            e = cudaGetLastError();
        }
        if (!e && best_E) e = launch_rescore64(ctx, L, G, best_geno, R, best_E, s);
        if (!e && evals_used) {
            evals_out_kernel<<<(R + 127) / 128, 128, 0, s>>>(ev, R, evals_used);
            ++ctx->launches;
            e = cudaGetLastError();
        }
        if (e) rc = cuda_err(ctx, e, "dock kernels");
    }
done:
    dev_free(ctx, popA, s);
    dev_free(ctx, popB, s);
    dev_free(ctx, EA, s);
    dev_free(ctx, EB, s);
    dev_free(ctx, picks, s);
    dev_free(ctx, ev, s);
    if (!best_E32) dev_free(ctx, bE32, s);
    return rc;
}

int dock(dock_ctx *ctx, const dock_grids *grids, const dock_ligand *lig, const dock_params *params, uint64_t seed,
         float *best_geno, double *best_E, int64_t *evals_used) {
    if (!ctx || !grids || !lig || !best_geno) return ctx ? set_err(ctx, DOCK_ERR_INVALID, "null argument") : DOCK_ERR_INVALID;
    dock_params P;
    int rc = resolve_params(ctx, params, P);
    if (rc) return rc;
    cudaStream_t s = nullptr;
    const int R = P.nruns, Gn = lig->dev.n_genes;
    float *g = (float *)dev_alloc(ctx, (size_t)R * Gn * 4, s);
    double *E = (double *)dev_alloc(ctx, (size_t)R * 8, s);
    int64_t *ev = (int64_t *)dev_alloc(ctx, (size_t)R * 8, s);
    if (!g || !E || !ev) {
        rc = set_err(ctx, DOCK_ERR_OOM, "device allocation failed in dock");
    } else {
        rc = dock_async(ctx, grids, lig, &P, seed, g, nullptr, E, ev, s);
        cudaError_t e = cudaSuccess;
        if (!rc) e = cudaMemcpyAsync(best_geno, g, (size_t)R * Gn * 4, cudaMemcpyDeviceToHost, s);
        if (!rc && !e && best_E) e = cudaMemcpyAsync(best_E, E, (size_t)R * 8, cudaMemcpyDeviceToHost, s);
        if (!rc && !e && evals_used) e = cudaMemcpyAsync(evals_used, ev, (size_t)R * 8, cudaMemcpyDeviceToHost, s);
        if (!rc && !e) e = cudaStreamSynchronize(s);
        if (!rc && e) rc = cuda_err(ctx, e, "dock copies");
    }
    dev_free(ctx, g, s);
    dev_free(ctx, E, s);
    dev_free(ctx, ev, s);
    return rc;
}

int dock_init_population(dock_ctx *ctx, const dock_grids *grids, int n_torsions, int pop, int nruns, uint64_t seed,
                         float *pop_out, void *stream) {
    if (!ctx || !grids || !pop_out || n_torsions < 0 || n_torsions > DOCK_MAX_TORSIONS || pop < 1 || nruns < 1)
        return ctx ? set_err(ctx, DOCK_ERR_INVALID, "invalid argument") : DOCK_ERR_INVALID;
    dock_params P;
    dock_default_params(&P);
    P.pop_size = pop;
    GaConst C = ga_const(P, n_torsions, nruns, seed);
    LigandDev l{};
    GridDev g = grids->dev;
    EvalLayout w = eval_layout(1, 1, 8, false, 1);
    float *no_e = nullptr;
    unsigned long long *no_ev = nullptr;
    void *a[] = {&l, &g, &C, &pop_out, &no_e, &no_ev, &w};
    cudaError_t e = launch_items(ctx, init_kernel<false>, pop * nruns, 4, (size_t)w.total * 16, (cudaStream_t)stream,
                                 "init_population", a);
    return e ? cuda_err(ctx, e, "init kernel") : DOCK_OK;
}

int dock_ga_children(dock_ctx *ctx, int n_torsions, int pop, int nruns, const float *pop_old, const float *E_old,
                     uint64_t seed, uint32_t generation, const dock_params *params, float *pop_new, int64_t *info,
                     void *stream) {
    if (!ctx || !pop_old || !E_old || !pop_new || n_torsions < 0 || n_torsions > DOCK_MAX_TORSIONS || pop < 2 ||
        nruns < 1)
        return ctx ? set_err(ctx, DOCK_ERR_INVALID, "invalid argument") : DOCK_ERR_INVALID;
    dock_params P;
    if (params) P = *params;
    else dock_default_params(&P);
    P.pop_size = pop;
    GaConst C = ga_const(P, n_torsions, nruns, seed);
    LigandDev l{};
    GridDev g{};
    EvalLayout w = eval_layout(1, 1, 8, false, 1);
    float *no_e = nullptr;
    unsigned long long *no_ev = nullptr;
    long long *inf = (long long *)info;
    const int *no_active = nullptr;
    void *a[] = {&l, &g, &C, &generation, &pop_old, &E_old, &pop_new, &no_e, &inf, &no_ev, &no_active, &w};
    cudaError_t e = launch_items(ctx, ga_kernel<false>, pop * nruns, 4, (size_t)w.total * 16, (cudaStream_t)stream,
                                 "ga_children", a);
    return e ? cuda_err(ctx, e, "ga kernel") : DOCK_OK;
}

int dock_ls_picks(dock_ctx *ctx, int pop, int n_ls, int nruns, uint64_t seed, uint32_t generation, int *picks,
                  void *stream) {
    if (!ctx || !picks || pop < 1 || n_ls < 0 || n_ls > pop || n_ls > kMaxLs || nruns < 1)
        return ctx ? set_err(ctx, DOCK_ERR_INVALID, "invalid argument") : DOCK_ERR_INVALID;
    if (n_ls == 0) return DOCK_OK;
    const uint2 key = make_uint2((uint32_t)seed, (uint32_t)(seed >> 32));
    picks_kernel<<<(nruns + 63) / 64, 64, 0, (cudaStream_t)stream>>>(pop, n_ls, nruns, key, generation, picks,
                                                                     nullptr);
    ++ctx->launches;
    cudaError_t e = cudaGetLastError();
    return e ? cuda_err(ctx, e, "picks kernel") : DOCK_OK;
}

int dock_local_search_trace(dock_ctx *ctx, const dock_grids *grids, const dock_ligand *lig, const float *x0, int B,
                            int iters, float rho, float eps, int threads, float *x_best, float *E_best,
                            float *x_trace, float *g_trace, float *E_trace, void *stream) {
    if (!ctx || !grids || !lig || (B > 0 && (!x0 || !x_best || !E_best)) || B < 0 || iters < 1 ||
        !(rho >= 0.f && rho < 1.f) || !(eps > 0.f))
        return ctx ? set_err(ctx, DOCK_ERR_INVALID, "invalid argument") : DOCK_ERR_INVALID;
    if ((x_trace || g_trace || E_trace) && !(x_trace && g_trace && E_trace))
        return set_err(ctx, DOCK_ERR_INVALID, "x_trace, g_trace and E_trace go together");
    int rc = check_maps(ctx, grids, lig);
    if (rc) return rc;
    if (B == 0) return DOCK_OK;
    const LigandDev &L = lig->dev;
    if (threads != 0 && threads != 32 && threads != 64 && threads != 128 && threads != 256)
        return set_err(ctx, DOCK_ERR_INVALID, "threads must be 0, 32, 64, 128 or 256");
    const int lw = ls_team_warps(ctx, B, threads, L);
    EvalLayout W = eval_layout(L.n_atoms, L.n_frag, L.nb8, true, lw);
    if (!evaluator_smem_ok(ctx, W, 1)) return set_err(ctx, DOCK_ERR_SIZE, "ligand too large for shared memory");
    LigandDev l = L;
    GridDev g = grids->dev;
    float *xin = const_cast<float *>(x0);
    float *no_pop = nullptr;
    const int *no_picks = nullptr;
    unsigned long long *no_ev = nullptr;
    int zero = 0, one = 1;
    LsTrace tr{x_trace, g_trace, E_trace};
    void *a[] = {&l,   &g,   &xin,    &no_pop, &no_picks, &zero, &one, &B,
                 &iters, &rho, &eps, &x_best, &E_best,   &no_ev, &W,   &tr};
    cudaError_t e = launch_ls(ctx, lw, B, W, (cudaStream_t)stream, "local_search", a);
    return e ? cuda_err(ctx, e, "local search kernel") : DOCK_OK;
}

int dock_local_search(dock_ctx *ctx, const dock_grids *grids, const dock_ligand *lig, const float *x0, int B,
                      int iters, float rho, float eps, int threads, float *x_best, float *E_best, void *stream) {
    return dock_local_search_trace(ctx, grids, lig, x0, B, iters, rho, eps, threads, x_best, E_best, nullptr,
                                   nullptr, nullptr, stream);
}

int dock_adadelta_step(dock_ctx *ctx, int B, int n_genes, float rho, float eps, float *x, const float *g,
                       float *Eg2, float *Edx2, void *stream) {
    if (!ctx || B < 0 || n_genes < 7 || n_genes > 7 + DOCK_MAX_TORSIONS || !(rho >= 0.f && rho < 1.f) || !(eps > 0.f) ||
        (B > 0 && (!x || !g || !Eg2 || !Edx2)))
        return ctx ? set_err(ctx, DOCK_ERR_INVALID, "invalid argument") : DOCK_ERR_INVALID;
    const long long n = (long long)B * n_genes;
    if (n == 0) return DOCK_OK;
    if (n > INT_MAX) return set_err(ctx, DOCK_ERR_INVALID, "B * n_genes exceeds INT_MAX");
    adadelta_step_kernel<<<(unsigned)((n + 255) / 256), 256, 0, (cudaStream_t)stream>>>((int)n, n_genes, rho, eps, x,
                                                                                       g, Eg2, Edx2);
    ++ctx->launches;
    cudaError_t e = cudaGetLastError();
    return e ? cuda_err(ctx, e, "ADADELTA step kernel") : DOCK_OK;
}

int dock_solis_wets(dock_ctx *ctx, const dock_grids *grids, const dock_ligand *lig, const float *x0,
                    const float *E0, int B, const dock_params *params, uint64_t seed, uint32_t run,
                    uint32_t generation, float *x_best, float *E_best, int64_t *evals, void *stream) {
    if (!ctx || !grids || !lig || B < 0 || (B > 0 && (!x0 || !x_best || !E_best)))
        return ctx ? set_err(ctx, DOCK_ERR_INVALID, "invalid argument") : DOCK_ERR_INVALID;
    dock_params P;
    if (params) P = *params;
    else dock_default_params(&P);
    P.ls_method = 1;
    if (P.ls_threads != 0 && P.ls_threads != 32 && P.ls_threads != 64 && P.ls_threads != 128 && P.ls_threads != 256)
        return set_err(ctx, DOCK_ERR_INVALID, "ls_threads must be 0, 32, 64, 128 or 256");
    if (P.ls_iters < 0) return set_err(ctx, DOCK_ERR_INVALID, "ls_iters must be >= 0");
    int rc = check_sw(ctx, P);
    if (rc) return rc;
    if ((rc = check_maps(ctx, grids, lig))) return rc;
    if (B == 0) return DOCK_OK;
    const LigandDev &L = lig->dev;
    const int lw = ls_team_warps(ctx, B, P.ls_threads, L);
    EvalLayout W = eval_layout(L.n_atoms, L.n_frag, L.nb8, false, lw);
    if (!evaluator_smem_ok(ctx, W, 1)) return set_err(ctx, DOCK_ERR_SIZE, "ligand too large for shared memory");
    LigandDev l = L;
    GridDev g = grids->dev;
    float *xin = const_cast<float *>(x0);
    float *no_pop = nullptr;
    const int *no_picks = nullptr, *no_active = nullptr;
    unsigned long long *no_ev = nullptr;
    long long *eo = (long long *)evals;
    int zero = 0, one = 1, iters = P.ls_iters;
    SwConst S = sw_const(P);
    uint2 key = make_uint2((uint32_t)seed, (uint32_t)(seed >> 32));
    void *a[] = {&l, &g, &xin, &no_pop, &no_picks, &zero, &one, &B, &iters, &S, &key, &run, &generation, &E0,
                 &x_best, &E_best, &no_ev, &eo, &no_active, &W};
    cudaError_t e = launch_sw(ctx, lw, B, W, (cudaStream_t)stream, "solis_wets", a);
    return e ? cuda_err(ctx, e, "Solis-Wets kernel") : DOCK_OK;
}

int dock_philox(dock_ctx *ctx, const uint32_t *ctr, int n, uint32_t key_lo, uint32_t key_hi, uint32_t *out,
                void *stream) {
    if (!ctx || n < 0 || (n > 0 && (!ctr || !out))) return ctx ? set_err(ctx, DOCK_ERR_INVALID, "invalid argument") : DOCK_ERR_INVALID;
    if (n == 0) return DOCK_OK;
    philox_kernel<<<(n + 255) / 256, 256, 0, (cudaStream_t)stream>>>(ctr, n, make_uint2(key_lo, key_hi), out);
    ++ctx->launches;
    cudaError_t e = cudaGetLastError();
    return e ? cuda_err(ctx, e, "philox kernel") : DOCK_OK;
}

}  // extern "C"

// ---------------------------------------------------------------------------
// Autotuning: device time of the local-search launch of dock() at a given
// team width, from the start points of an initial population.

int tune_ls_launch(dock_ctx *ctx, const dock_grids *grids, const dock_ligand *lig, const dock_params &P0,
                   int threads, int reps, double *ms) {
    *ms = -1.0;
    dock_params P;
    int rc = resolve_params(ctx, &P0, P);
    if (rc) return rc;
    if ((rc = check_maps(ctx, grids, lig))) return rc;
    const LigandDev &L = lig->dev;
    int chains = P.nruns * P.ls_count;
    if (chains <= 0 || P.ls_iters <= 0) {
        *ms = 0.0;
        return DOCK_OK;
    }
    const int W = ls_team_warps(ctx, chains, threads, L);
    if (32 * W != threads) return DOCK_OK;  // does not fit shared memory
    const bool sw = P.ls_method == 1;
    EvalLayout Y = eval_layout(L.n_atoms, L.n_frag, L.nb8, !sw, W);
    EvalLayout Wn = eval_layout(L.n_atoms, L.n_frag, L.nb8, false, 1);
    if (!evaluator_smem_ok(ctx, Y, 1)) return DOCK_OK;
    const int Gn = L.n_genes;
    int iters = std::min(P.ls_iters, 50);
    cudaStream_t s = nullptr;
    float *x = (float *)dev_alloc(ctx, (size_t)chains * Gn * 4, s);
    float *xo = (float *)dev_alloc(ctx, (size_t)chains * Gn * 4, s);
    float *E0 = (float *)dev_alloc(ctx, (size_t)chains * 4, s);
    float *Eo = (float *)dev_alloc(ctx, (size_t)chains * 4, s);
    unsigned long long *cnt = (unsigned long long *)dev_alloc(ctx, 8, s);
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    cudaError_t e = cudaSuccess;
    if (!x || !xo || !E0 || !Eo || !cnt) {
        rc = set_err(ctx, DOCK_ERR_OOM, "dock_tune: allocation failed");
    } else {
        dock_params Q = P;
        Q.pop_size = chains;
        GaConst C = ga_const(Q, L.n_tors, 1, 0x7475u);
        LigandDev l = L;
        GridDev g = grids->dev;
        void *a[] = {&l, &g, &C, &x, &E0, &cnt, &Wn};
        e = launch_items(ctx, init_kernel<true>, chains, 1, (size_t)Wn.total * 4, s, "tune_init", a);
        float *no_pop = nullptr;
        const int *no_picks = nullptr, *no_active = nullptr;
        unsigned long long *no_ev = nullptr;
        long long *no_eo = nullptr;
        int zero = 0, one = 1;
        float rho = P.rho, eps = P.eps;
        SwConst S = sw_const(P);
        uint2 key = make_uint2(1u, 2u);
        uint32_t run0 = 0, gen0 = 0;
        const float *e0p = E0;
        LsTrace no_trace{nullptr, nullptr, nullptr};
        void *la[] = {&l,  &g,  &x,     &no_pop, &no_picks, &zero, &one, &chains, &iters,
                      &rho, &eps, &xo, &Eo,    &no_ev,    &Y,    &no_trace};
        void *sa[] = {&l, &g, &x, &no_pop, &no_picks, &zero, &one, &chains, &iters, &S, &key, &run0, &gen0, &e0p,
                      &xo, &Eo, &no_ev, &no_eo, &no_active, &Y};
        auto one_launch = [&]() {
            return sw ? launch_sw(ctx, W, chains, Y, s, "tune_ls", sa) : launch_ls(ctx, W, chains, Y, s, "tune_ls", la);
        };
        if (!e) e = one_launch();
        if (!e) e = cudaEventCreate(&e0);
        if (!e) e = cudaEventCreate(&e1);
        if (!e) e = cudaEventRecord(e0, s);
        for (int r = 0; r < reps && !e; ++r) e = one_launch();
        if (!e) e = cudaEventRecord(e1, s);
        if (!e) e = cudaEventSynchronize(e1);
        float t = 0.f;
        if (!e) e = cudaEventElapsedTime(&t, e0, e1);
        if (e) rc = cuda_err(ctx, e, "dock_tune local search");
        else *ms = (double)t / reps;
    }
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    dev_free(ctx, x, s);
    dev_free(ctx, xo, s);
    dev_free(ctx, E0, s);
    dev_free(ctx, Eo, s);
    dev_free(ctx, cnt, s);
    return rc;
}

// Device time of score_grad_batch over an initial population of
// params.pop_size * nruns genotypes at register cap `mb`.
int tune_score_launch(dock_ctx *ctx, const dock_grids *grids, const dock_ligand *lig, const dock_params &P, int mb,
                      int reps, double *ms) {
    *ms = -1.0;
    int rc = check_maps(ctx, grids, lig);
    if (rc) return rc;
    const LigandDev &L = lig->dev;
    const int B = P.pop_size * P.nruns, Gn = L.n_genes;
    if (B < 1) return set_err(ctx, DOCK_ERR_INVALID, "dock_tune: empty batch");
    cudaStream_t s = nullptr;
    float *x = (float *)dev_alloc(ctx, (size_t)B * Gn * 4, s);
    float *E = (float *)dev_alloc(ctx, (size_t)B * 4, s);
    float *g = (float *)dev_alloc(ctx, (size_t)B * Gn * 4, s);
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    const int keep = ctx->score_min_blocks;
    cudaError_t e = cudaSuccess;
    if (!x || !E || !g) {
        rc = set_err(ctx, DOCK_ERR_OOM, "dock_tune: allocation failed");
    } else {
        dock_params Q = P;
        Q.pop_size = B;
        GaConst C = ga_const(Q, L.n_tors, 1, 0x7475u);
        LigandDev l{};
        l.n_tors = L.n_tors;
        GridDev gd = grids->dev;
        EvalLayout w = eval_layout(1, 1, 8, false, 1);
        float *no_e = nullptr;
        unsigned long long *no_ev = nullptr;
        void *a[] = {&l, &gd, &C, &x, &no_e, &no_ev, &w};
        e = launch_items(ctx, init_kernel<false>, B, 4, (size_t)w.total * 16, s, "tune_init", a);
        ctx->score_min_blocks = mb;
        if (!e) e = launch_score(ctx, L, grids->dev, x, B, E, g, s);
        if (!e) e = cudaEventCreate(&e0);
        if (!e) e = cudaEventCreate(&e1);
        if (!e) e = cudaEventRecord(e0, s);
        for (int r = 0; r < reps && !e; ++r) e = launch_score(ctx, L, grids->dev, x, B, E, g, s);
        if (!e) e = cudaEventRecord(e1, s);
        if (!e) e = cudaEventSynchronize(e1);
        float t = 0.f;
        if (!e) e = cudaEventElapsedTime(&t, e0, e1);
        ctx->score_min_blocks = keep;
        if (e) rc = cuda_err(ctx, e, "dock_tune score");
        else *ms = (double)t / reps;
    }
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    dev_free(ctx, x, s);
    dev_free(ctx, E, s);
    dev_free(ctx, g, s);
    return rc;
}

extern "C" int dock_tune(dock_ctx *ctx, const dock_grids *grids, const dock_ligand *const *ligs, int n_ligs,
                         const dock_params *params, int what, const int *cand, int n_cand, int reps, double *ms) {
    if (!ctx) return DOCK_ERR_INVALID;
    if (!grids || !ligs || n_ligs < 1 || !cand || n_cand < 1 || reps < 1 || !ms)
        return set_err(ctx, DOCK_ERR_INVALID, "dock_tune: invalid argument");
    for (int k = 0; k < n_ligs; ++k)
        if (!ligs[k]) return set_err(ctx, DOCK_ERR_INVALID, "dock_tune: null ligand");
    dock_params P;
    if (params) P = *params;
    else dock_default_params(&P);
    for (int i = 0; i < n_cand; ++i) {
        const int c = cand[i];
        int rc = DOCK_OK;
        if (what == DOCK_TUNE_LS_THREADS) {
            if (c != 32 && c != 64 && c != 128 && c != 256)
                return set_err(ctx, DOCK_ERR_INVALID, "dock_tune: threads must be 32, 64, 128 or 256");
            rc = tune_ls_launch(ctx, grids, ligs[0], P, c, reps, &ms[i]);
        } else if (what == DOCK_TUNE_BATCH_WARPS) {
            if (c != 1 && c != 2 && c != 4) return set_err(ctx, DOCK_ERR_INVALID, "dock_tune: warps must be 1, 2 or 4");
            ms[i] = -1.0;
            rc = tune_batch_launch(ctx, grids, ligs, n_ligs, P, c, 0, reps, &ms[i]);
            if (rc == DOCK_ERR_SIZE) {  // this width does not fit: reported as -1
                ms[i] = -1.0;
                rc = DOCK_OK;
            }
        } else if (what == DOCK_TUNE_BATCH_BLOCKS) {
            if (c != 3 && c != 4) return set_err(ctx, DOCK_ERR_INVALID, "dock_tune: batch blocks must be 3 or 4");
            ms[i] = -1.0;
            rc = tune_batch_launch(ctx, grids, ligs, n_ligs, P, 0, c, reps, &ms[i]);
            if (rc == DOCK_ERR_SIZE) {
                ms[i] = -1.0;
                rc = DOCK_OK;
            }
        } else if (what == DOCK_TUNE_SCORE_BLOCKS) {
            if (c != 1 && c != 6 && c != 8) return set_err(ctx, DOCK_ERR_INVALID, "dock_tune: blocks must be 1, 6 or 8");
            rc = tune_score_launch(ctx, grids, ligs[0], P, c, reps, &ms[i]);
        } else {
            return set_err(ctx, DOCK_ERR_INVALID, "dock_tune: unknown kernel family");
        }
        if (rc) return rc;
    }
    return DOCK_OK;
}

// ---------------------------------------------------------------------------
// dock_async_noalloc: the docking of dock_async with its working buffers
// (two populations, their energies, the local-search picks and the per-run
// evaluation counters) carved out of one fixed device array instead of
// allocated memory.

namespace {

// Module-scope scratch: every device that loads the library holds one copy
// until the process exits.
__device__ __align__(256) unsigned char g_noalloc_scratch[DOCK_NOALLOC_SCRATCH_BYTES];

// Device address of the array on each device, looked up once per device
// with that device current (the host-side name is only a stand-in).
std::mutex g_noalloc_mu;
void *g_noalloc_ptr[128] = {};

int noalloc_base(dock_ctx *ctx, unsigned char **base) {
    int cur = -1;
    cudaError_t e = cudaGetDevice(&cur);
    if (e != cudaSuccess) return cuda_err(ctx, e, "cudaGetDevice");
    if (cur != ctx->device || cur < 0 || cur >= 128)
        return set_err(ctx, DOCK_ERR_INVALID, "the context's device must be the current device");
    std::lock_guard<std::mutex> g(g_noalloc_mu);
    if (!g_noalloc_ptr[cur]) {
        void *p = nullptr;
        e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess || !p) return cuda_err(ctx, e == cudaSuccess ? cudaErrorInvalidSymbol : e, "cudaGetSymbolAddress");
        g_noalloc_ptr[cur] = p;
    }
    *base = (unsigned char *)g_noalloc_ptr[cur];
    return DOCK_OK;
}

size_t align256(size_t v) { return (v + 255) & ~(size_t)255; }

}  // namespace

// Called by dock_create with the context's device current: the lookup loads
// this file's device code (modules load lazily), so the array exists from the
// context's creation on and a later dock_async_noalloc allocates nothing.
int noalloc_prepare(dock_ctx *ctx) {
    unsigned char *base = nullptr;
    return noalloc_base(ctx, &base);
}

extern "C" int dock_async_noalloc(dock_ctx *ctx, const dock_grids *grids, const dock_ligand *lig,
                                  const dock_params *params, uint64_t seed, float *best_geno, float *best_E32,
                                  double *best_E, int64_t *evals_used, void *stream) {
    if (!ctx || !grids || !lig || !best_geno) return ctx ? set_err(ctx, DOCK_ERR_INVALID, "null argument") : DOCK_ERR_INVALID;
    dock_params P;
    int rc = resolve_params(ctx, params, P);
    if (rc) return rc;
    if (P.ls_method != 0) return set_err(ctx, DOCK_ERR_INVALID, "dock_async_noalloc runs the ADADELTA search only");
    if ((rc = check_maps(ctx, grids, lig))) return rc;
    cudaStream_t s = (cudaStream_t)stream;
    const LigandDev &L = lig->dev;
    const GridDev &G = grids->dev;
    const int Gn = L.n_genes, pop = P.pop_size, R = P.nruns, nls = P.ls_count;
    const EvalLayout Wn = eval_layout(L.n_atoms, L.n_frag, L.nb8, false, 1);
    const int lw = ls_team_warps(ctx, P.nruns * P.ls_count, P.ls_threads, L);
    const EvalLayout Wg = eval_layout(L.n_atoms, L.n_frag, L.nb8, true, lw);
    if (!evaluator_smem_ok(ctx, Wg, 1)) return set_err(ctx, DOCK_ERR_SIZE, "ligand too large for shared memory");
    const int gw = evaluator_smem_ok(ctx, Wn, 4) ? 4 : 1;
    const size_t items = (size_t)R * pop;
    // carve the scratch: populations, energies, picks, counters, FP32 bests
    const size_t o_popA = 0, o_popB = o_popA + align256(items * Gn * 4);
    const size_t o_EA = o_popB + align256(items * Gn * 4), o_EB = o_EA + align256(items * 4);
    const size_t o_picks = o_EB + align256(items * 4);
    const size_t o_ev = o_picks + align256((size_t)R * (nls > 0 ? nls : 1) * 4);
    const size_t o_bE = o_ev + align256((size_t)R * 8);
    const size_t need = o_bE + (best_E32 ? 0 : align256((size_t)R * 4));
    if (need > (size_t)DOCK_NOALLOC_SCRATCH_BYTES)
        return set_err(ctx, DOCK_ERR_SIZE, "dock_async_noalloc needs " + std::to_string(need) +
                                               " bytes of scratch; its fixed array holds " +
                                               std::to_string((size_t)DOCK_NOALLOC_SCRATCH_BYTES));
    unsigned char *base = nullptr;
    if ((rc = noalloc_base(ctx, &base))) return rc;
    float *popA = (float *)(base + o_popA), *popB = (float *)(base + o_popB);
    float *EA = (float *)(base + o_EA), *EB = (float *)(base + o_EB);
    int *picks = (int *)(base + o_picks);
    unsigned long long *ev = (unsigned long long *)(base + o_ev);
    float *bE32 = best_E32 ? best_E32 : (float *)(base + o_bE);
    GaConst C = ga_const(P, L.n_tors, R, seed);
    LigandDev l = L;
    GridDev g = G;
    EvalLayout wn = Wn, wg = Wg;
    // the array keeps the previous call's contents: the counters restart at 0
    cudaError_t e = cudaMemsetAsync(ev, 0, (size_t)R * 8, s);
    {
        void *a[] = {&l, &g, &C, &popA, &EA, &ev, &wn};
        if (!e) e = launch_items(ctx, init_kernel<true>, (int)items, gw, (size_t)Wn.total * 4 * gw, s, "dock_init", a);
    }
    const long long per_gen = (long long)(pop - 1) + (long long)nls * P.ls_iters;
    long long ngen = 0;
    if (P.max_evals > pop) ngen = (P.max_evals - pop + per_gen - 1) / per_gen;
    const int chains = R * nls;
    long long *no_info = nullptr;
    float *no_out = nullptr;
    for (long long gen = 1; gen <= ngen && !e; ++gen) {
        uint32_t g32 = (uint32_t)gen;
        const int *no_active = nullptr;
        void *a[] = {&l, &g, &C, &g32, &popA, &EA, &popB, &EB, &no_info, &ev, &no_active, &wn};
        e = launch_items(ctx, ga_kernel<true>, (int)items, gw, (size_t)Wn.total * 4 * gw, s, "dock_ga", a);
        if (!e && chains > 0 && P.ls_iters > 0) {
            picks_kernel<<<(R + 63) / 64, 64, 0, s>>>(pop, nls, R, C.key, g32, picks, nullptr);
            ++ctx->launches;
            e = cudaGetLastError();
            int iters = P.ls_iters;
            float rho = P.rho, eps = P.eps;
            int nl = nls, ch = chains, popn = pop;
            LsTrace no_trace{nullptr, nullptr, nullptr};
            void *c[] = {&l,   &g,   &popB,   &EB,     &picks, &popn, &nl,      &ch,
                         &iters, &rho, &eps, &no_out, &no_out, &ev,   &wg,  &no_trace};
            if (!e) e = launch_ls(ctx, lw, chains, Wg, s, "dock_ls", c);
        }
        std::swap(popA, popB);
        std::swap(EA, EB);
    }
    if (!e) {
        final_kernel<<<(R + 3) / 4, 128, 0, s>>>(popA, EA, pop, R, Gn, best_geno, bE32);
        ++ctx->launches;
        e = cudaGetLastError();
    }
    if (!e && best_E) e = launch_rescore64(ctx, L, G, best_geno, R, best_E, s);
    if (!e && evals_used) {
        evals_out_kernel<<<(R + 127) / 128, 128, 0, s>>>(ev, R, evals_used);
        ++ctx->launches;
        e = cudaGetLastError();
    }
    return e ? cuda_err(ctx, e, "dock kernels") : DOCK_OK;
}
