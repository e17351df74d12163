// host.cpp -- context, memory, errors, tracing, ligand preprocessing and
// grid loading of libdock.so.
#include <math.h>
#include <string.h>

#include <algorithm>
#include <cmath>
#include <queue>
#include <string>
#include <vector>

#include "forcefield.h"
#include "internal.h"

// ---------------------------------------------------------------------------
// errors, memory, tracing

int set_err(dock_ctx *ctx, int code, const std::string &msg) {
    if (ctx) ctx->err = msg;
    return code;
}

int cuda_err(dock_ctx *ctx, cudaError_t e, const char *what) {
    return set_err(ctx, e == cudaErrorMemoryAllocation ? DOCK_ERR_OOM : DOCK_ERR_CUDA,
                   std::string(what) + ": " + cudaGetErrorString(e));
}

void *dev_alloc(dock_ctx *ctx, size_t bytes, cudaStream_t s) {
    if (bytes == 0) bytes = 16;
    if (ctx->has_alloc) return ctx->alloc.alloc(bytes, (void *)s, ctx->alloc.user);
    void *p = nullptr;
    if (cudaMallocAsync(&p, bytes, s) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    return p;
}

// Solis-Wets constants: finite, positive scales, at least one step in a
// run, and iteration indices that fit the 16-bit draw field (10 it + 9).
int check_sw(dock_ctx *ctx, const dock_params &p) {
    if (p.ls_method != 0 && p.ls_method != 1) return set_err(ctx, DOCK_ERR_INVALID, "ls_method must be 0 or 1");
    if (p.ls_method == 0) return DOCK_OK;
    const bool ok = p.ls_iters <= 6553 && std::isfinite(p.sw_rho0) && p.sw_rho0 > 0.f && p.sw_rho_lo >= 0.f &&
                    std::isfinite(p.sw_expand) && p.sw_expand > 0.f && p.sw_contract > 0.f && p.sw_contract < 1.f &&
                    p.sw_succ >= 1 && p.sw_fail >= 1 && std::isfinite(p.sw_step[0]) && std::isfinite(p.sw_step[1]) &&
                    std::isfinite(p.sw_step[2]) && p.sw_step[0] >= 0.f && p.sw_step[1] >= 0.f && p.sw_step[2] >= 0.f;
    return ok ? DOCK_OK : set_err(ctx, DOCK_ERR_INVALID, "invalid Solis-Wets parameters (ls_iters <= 6553)");
}

long long *host_status(dock_ctx *ctx) {
    if (!ctx->h_status && cudaHostAlloc((void **)&ctx->h_status, 2 * sizeof(long long), cudaHostAllocDefault)) {
        cudaGetLastError();
        ctx->h_status = nullptr;
    }
    return ctx->h_status;
}

void dev_free(dock_ctx *ctx, void *p, cudaStream_t s) {
    if (!p) return;
    if (ctx->has_alloc) ctx->alloc.free(p, (void *)s, ctx->alloc.user);
    else cudaFreeAsync(p, s);
}

int kernel_id(dock_ctx *ctx, const char *name) {
    for (size_t i = 0; i < ctx->kernel_names.size(); ++i)
        if (ctx->kernel_names[i] == name) return (int)i;
    ctx->kernel_names.emplace_back(name);
    ctx->kernel_ms.push_back(0.0);
    ctx->kernel_launches.push_back(0);
    return (int)ctx->kernel_names.size() - 1;
}

static cudaEvent_t pool_event(dock_ctx *ctx) {
    if (!ctx->event_pool.empty()) {
        cudaEvent_t e = ctx->event_pool.back();
        ctx->event_pool.pop_back();
        return e;
    }
    cudaEvent_t e = nullptr;
    cudaEventCreate(&e);
    return e;
}

void timing_begin(dock_ctx *ctx, int kid, cudaStream_t s, TimedLaunch *tl) {
    tl->kernel = -1;
    if (!ctx->timing) return;
    tl->kernel = kid;
    tl->start = pool_event(ctx);
    tl->stop = pool_event(ctx);
    cudaEventRecord(tl->start, s);
}

void timing_end(dock_ctx *ctx, cudaStream_t s, TimedLaunch *tl) {
    if (tl->kernel < 0) return;
    cudaEventRecord(tl->stop, s);
    ctx->pending.push_back(*tl);
}

static void flush_timing(dock_ctx *ctx, bool keep) {
    for (const TimedLaunch &t : ctx->pending) {
        float ms = 0.f;
        if (cudaEventSynchronize(t.stop) == cudaSuccess && cudaEventElapsedTime(&ms, t.start, t.stop) == cudaSuccess &&
            keep) {
            ctx->kernel_ms[t.kernel] += ms;
            ctx->kernel_launches[t.kernel] += 1;
        }
        ctx->event_pool.push_back(t.start);
        ctx->event_pool.push_back(t.stop);
    }
    ctx->pending.clear();
}

int check_maps(dock_ctx *ctx, const dock_grids *g, const dock_ligand *l) {
    for (int t : l->types)
        if (g->map_of_type[t] < 0) return set_err(ctx, DOCK_ERR_NOMAP, "ligand atom type without a map");
    return DOCK_OK;
}

extern "C" {

int dock_version(void) { return 100; }

void dock_default_params(dock_params *p) {
    if (!p) return;
    p->pop_size = 150;
    p->nruns = 10;
    p->max_evals = 100000;
    p->ls_count = -1;
    p->ls_iters = 100;
    p->rho = 0.8f;
    p->eps = 1e-2f;
    p->p_tour = 0.6f;
    p->p_cross = 0.8f;
    p->p_mut = 0.02f;
    p->trans_mut = 2.0f;
    p->ls_threads = 0;
    p->ls_method = 0;
    p->sw_rho0 = 1.0f;
    p->sw_rho_lo = 0.01f;
    p->sw_expand = 2.0f;
    p->sw_contract = 0.5f;
    p->sw_succ = 4;
    p->sw_fail = 4;
    p->sw_step[0] = 1.0f;
    p->sw_step[1] = 0.2f;
    p->sw_step[2] = 0.75f;
    p->batch_warps = 0;
    p->batch_pack = 0;
}

int dock_create(dock_ctx **out, int device, const dock_allocator *alloc) {
    if (!out) return DOCK_ERR_INVALID;
    *out = nullptr;
    int n = 0;
    if (cudaGetDeviceCount(&n) != cudaSuccess || device < 0 || device >= n) {
        cudaGetLastError();
        return DOCK_ERR_CUDA;
    }
    if (cudaSetDevice(device) != cudaSuccess) return DOCK_ERR_CUDA;
    dock_ctx *c = new dock_ctx();
    c->device = device;
    cudaDeviceGetAttribute(&c->num_sms, cudaDevAttrMultiProcessorCount, device);
    int optin = 0;
    cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, device);
    c->smem_optin = (size_t)optin;
    if (alloc && alloc->alloc && alloc->free) {
        c->alloc = *alloc;
        c->has_alloc = true;
    }
    // the no-allocation docking's array comes into being here, not in its
    // first call; a failure is left for that call to report
    if (noalloc_prepare(c) != DOCK_OK) cudaGetLastError();
    *out = c;
    return DOCK_OK;
}

int dock_destroy(dock_ctx *ctx) {
    if (!ctx) return DOCK_ERR_INVALID;
    flush_timing(ctx, false);
    for (cudaEvent_t e : ctx->event_pool) cudaEventDestroy(e);
    if (ctx->h_status) cudaFreeHost(ctx->h_status);
    delete ctx;
    return DOCK_OK;
}

int dock_set_option(dock_ctx *ctx, int option, int value) {
    if (!ctx) return DOCK_ERR_INVALID;
    if (option == DOCK_OPT_SCORE_BLOCKS) {
        if (value != 1 && value != 6 && value != 8) return set_err(ctx, DOCK_ERR_INVALID, "score blocks must be 1, 6 or 8");
        ctx->score_min_blocks = value;
        return DOCK_OK;
    }
    if (option == DOCK_OPT_BATCH_BLOCKS) {
        if (value != 3 && value != 4) return set_err(ctx, DOCK_ERR_INVALID, "batch blocks must be 3 or 4");
        ctx->batch_min_blocks = value;
        return DOCK_OK;
    }
    return set_err(ctx, DOCK_ERR_INVALID, "unknown option");
}

int dock_get_option(const dock_ctx *ctx, int option, int *value) {
    if (!ctx || !value) return DOCK_ERR_INVALID;
    if (option == DOCK_OPT_SCORE_BLOCKS) {
        *value = ctx->score_min_blocks;
        return DOCK_OK;
    }
    if (option == DOCK_OPT_BATCH_BLOCKS) {
        *value = ctx->batch_min_blocks;
        return DOCK_OK;
    }
    return DOCK_ERR_INVALID;
}

const char *dock_last_error(const dock_ctx *ctx) { return ctx ? ctx->err.c_str() : "null context"; }

int dock_set_timing(dock_ctx *ctx, int enable) {
    if (!ctx) return DOCK_ERR_INVALID;
    ctx->timing = enable != 0;
    return DOCK_OK;
}

int dock_reset_timing(dock_ctx *ctx) {
    if (!ctx) return DOCK_ERR_INVALID;
    flush_timing(ctx, false);
    std::fill(ctx->kernel_ms.begin(), ctx->kernel_ms.end(), 0.0);
    std::fill(ctx->kernel_launches.begin(), ctx->kernel_launches.end(), 0);
    return DOCK_OK;
}

int dock_kernel_time(dock_ctx *ctx, const char *kernel, double *total_ms, int64_t *launches) {
    if (!ctx || !kernel) return DOCK_ERR_INVALID;
    flush_timing(ctx, true);
    const int k = kernel_id(ctx, kernel);
    if (total_ms) *total_ms = ctx->kernel_ms[k];
    if (launches) *launches = ctx->kernel_launches[k];
    return DOCK_OK;
}

int64_t dock_launch_count(const dock_ctx *ctx) { return ctx ? ctx->launches : -1; }

// ---------------------------------------------------------------------------
// grids

static int finish_grids(dock_ctx *ctx, dock_grids *g, const int dims[3], const double origin[3], double spacing,
                        cudaStream_t s) {
    GridDev &d = g->dev;
    d.nx = dims[0];
    d.ny = dims[1];
    d.nz = dims[2];
    d.M = g->n_maps;
    d.ox = (float)origin[0];
    d.oy = (float)origin[1];
    d.oz = (float)origin[2];
    d.h = (float)spacing;
    d.inv_h = (float)(1.0 / spacing);
    d.ox64 = origin[0];
    d.oy64 = origin[1];
    d.oz64 = origin[2];
    d.h64 = spacing;
    for (int a = 0; a < 3; ++a) {
        d.box_lo[a] = (float)origin[a];
        d.box_len[a] = (float)((dims[a] - 1) * spacing);
    }
    d.emap = d.dmap = -1;
    for (int m = 0; m < g->n_maps; ++m) {
        const int t = g->map_type[m];
        if (t == DOCK_MAP_ELEC) d.emap = m;
        else if (t == DOCK_MAP_DESOLV) d.dmap = m;
        else g->map_of_type[t] = m;
    }
    d.mstride = (long long)(d.nx - 1) * (d.ny - 1) * d.nz;
    g->cells_mem = dev_alloc(ctx, (size_t)d.mstride * d.M * 16, s);
    g->lut_mem = dev_alloc(ctx, 8 * sizeof(int), s);
    if (!g->cells_mem || !g->lut_mem) return set_err(ctx, DOCK_ERR_OOM, "grid allocation failed");
    d.cells = (const float4 *)g->cells_mem;
    d.map_of_type = (const int *)g->lut_mem;
    cudaError_t e = cudaMemcpyAsync(g->lut_mem, g->map_of_type, 8 * sizeof(int), cudaMemcpyHostToDevice, s);
    if (!e) e = launch_relayout(d, (float4 *)g->cells_mem, s);
    if (!e) e = cudaStreamSynchronize(s);
    if (e) return cuda_err(ctx, e, "grid upload");
    return DOCK_OK;
}

static int check_box(dock_ctx *ctx, const int dims[3], const double origin[3], double spacing) {
    if (!dims || !origin) return set_err(ctx, DOCK_ERR_INVALID, "null grid geometry");
    for (int a = 0; a < 3; ++a)
        if (dims[a] < 2 || dims[a] > 4096 || !isfinite(origin[a]))
            return set_err(ctx, DOCK_ERR_INVALID, "grid dims must be in 2..4096 and the origin finite");
    if (!(spacing > 0.0) || !isfinite(spacing)) return set_err(ctx, DOCK_ERR_INVALID, "spacing must be > 0");
    return DOCK_OK;
}

int load_grids(dock_ctx *ctx, const float *maps, int n_maps, const int dims[3], const double origin[3], double spacing,
               const int *map_type, dock_grids **out) {
    if (!ctx || !out) return DOCK_ERR_INVALID;
    *out = nullptr;
    int rc = check_box(ctx, dims, origin, spacing);
    if (rc) return rc;
    if (!maps || !map_type || n_maps < 3 || n_maps > DOCK_NTYPES + 2)
        return set_err(ctx, DOCK_ERR_INVALID, "need 3..9 maps");
    int ne = 0, nd = 0, seen[DOCK_NTYPES] = {0};
    for (int m = 0; m < n_maps; ++m) {
        const int t = map_type[m];
        if (t == DOCK_MAP_ELEC) ++ne;
        else if (t == DOCK_MAP_DESOLV) ++nd;
        else if (t < 0 || t >= DOCK_NTYPES || seen[t]++) return set_err(ctx, DOCK_ERR_INVALID, "bad or repeated map type");
    }
    if (ne != 1 || nd != 1) return set_err(ctx, DOCK_ERR_INVALID, "need exactly one electrostatic and one desolvation map");
    const size_t nn = (size_t)dims[0] * dims[1] * dims[2];
    for (size_t i = 0; i < nn * n_maps; ++i)
        if (!isfinite(maps[i])) return set_err(ctx, DOCK_ERR_INVALID, "non-finite map value");
    dock_grids *g = new dock_grids();
    g->n_maps = n_maps;
    g->map_type.assign(map_type, map_type + n_maps);
    cudaStream_t s = nullptr;
    g->nodes_mem = dev_alloc(ctx, nn * n_maps * 4, s);
    if (!g->nodes_mem) {
        free_grids(ctx, g);
        return set_err(ctx, DOCK_ERR_OOM, "grid allocation failed");
    }
    g->dev.nodes = (const float *)g->nodes_mem;
    cudaError_t e = cudaMemcpyAsync(g->nodes_mem, maps, nn * n_maps * 4, cudaMemcpyHostToDevice, s);
    if (e) {
        free_grids(ctx, g);
        return cuda_err(ctx, e, "grid upload");
    }
    rc = finish_grids(ctx, g, dims, origin, spacing, s);
    if (rc) {
        free_grids(ctx, g);
        return rc;
    }
    *out = g;
    return DOCK_OK;
}

int build_grids(dock_ctx *ctx, int n_rec, const double *rxyz, const int *rtype, const double *rq, const int dims[3],
                const double origin[3], double spacing, int n_type_maps, const int *map_types, dock_grids **out) {
    if (!ctx || !out) return DOCK_ERR_INVALID;
    *out = nullptr;
    int rc = check_box(ctx, dims, origin, spacing);
    if (rc) return rc;
    if (n_rec < 1 || !rxyz || !rtype || !rq || n_type_maps < 1 || n_type_maps > DOCK_NTYPES || !map_types)
        return set_err(ctx, DOCK_ERR_INVALID, "bad receptor or map list");
    int seen[DOCK_NTYPES] = {0};
    for (int m = 0; m < n_type_maps; ++m)
        if (map_types[m] < 0 || map_types[m] >= DOCK_NTYPES || seen[map_types[m]]++)
            return set_err(ctx, DOCK_ERR_INVALID, "bad or repeated map type");
    std::vector<float4> rec(n_rec);
    for (int j = 0; j < n_rec; ++j) {
        if (rtype[j] < 0 || rtype[j] >= DOCK_NTYPES) return set_err(ctx, DOCK_ERR_TYPE, "unknown receptor atom type");
        rec[j] = make_float4((float)(rxyz[3 * j] - origin[0]), (float)(rxyz[3 * j + 1] - origin[1]),
                             (float)(rxyz[3 * j + 2] - origin[2]), (float)rq[j]);
    }
    dock_grids *g = new dock_grids();
    g->n_maps = n_type_maps + 2;
    g->map_type.assign(map_types, map_types + n_type_maps);
    g->map_type.push_back(DOCK_MAP_ELEC);
    g->map_type.push_back(DOCK_MAP_DESOLV);
    cudaStream_t s = nullptr;
    const size_t nn = (size_t)dims[0] * dims[1] * dims[2];
    g->nodes_mem = dev_alloc(ctx, nn * g->n_maps * 4, s);
    float4 *drec = (float4 *)dev_alloc(ctx, n_rec * sizeof(float4), s);
    int *dt = (int *)dev_alloc(ctx, n_rec * sizeof(int), s);
    cudaError_t e = cudaSuccess;
    if (!g->nodes_mem || !drec || !dt) {
        rc = set_err(ctx, DOCK_ERR_OOM, "grid allocation failed");
    } else {
        g->dev.nodes = (const float *)g->nodes_mem;
        e = cudaMemcpyAsync(drec, rec.data(), n_rec * sizeof(float4), cudaMemcpyHostToDevice, s);
        if (!e) e = cudaMemcpyAsync(dt, rtype, n_rec * sizeof(int), cudaMemcpyHostToDevice, s);
        if (!e) e = launch_build_maps(n_rec, drec, dt, dims[0], dims[1], dims[2], spacing, n_type_maps, map_types,
                                      (float *)g->nodes_mem, s);
        if (!e) ++ctx->launches;
        if (!e) e = cudaStreamSynchronize(s);
        if (e) rc = cuda_err(ctx, e, "map builder");
    }
    dev_free(ctx, drec, s);
    dev_free(ctx, dt, s);
    if (!rc) rc = finish_grids(ctx, g, dims, origin, spacing, s);
    if (rc) {
        free_grids(ctx, g);
        return rc;
    }
    *out = g;
    return DOCK_OK;
}

int grids_read_maps(dock_ctx *ctx, const dock_grids *g, float *maps_out) {
    if (!ctx || !g || !maps_out) return DOCK_ERR_INVALID;
    const size_t n = (size_t)g->dev.nx * g->dev.ny * g->dev.nz * g->n_maps;
    cudaError_t e = cudaMemcpy(maps_out, g->nodes_mem, n * 4, cudaMemcpyDeviceToHost);
    return e ? cuda_err(ctx, e, "grid download") : DOCK_OK;
}

int free_grids(dock_ctx *ctx, dock_grids *g) {
    if (!ctx || !g) return DOCK_ERR_INVALID;
    cudaStreamSynchronize(nullptr);
    dev_free(ctx, g->cells_mem, nullptr);
    dev_free(ctx, g->nodes_mem, nullptr);
    dev_free(ctx, g->lut_mem, nullptr);
    delete g;
    return DOCK_OK;
}

}  // extern "C"

// ---------------------------------------------------------------------------
// ligand preprocessing

namespace {

struct Blob {
    std::vector<unsigned char> bytes;
    size_t add(const void *p, size_t n) {
        size_t off = (bytes.size() + 15) & ~(size_t)15;
        bytes.resize(off + (n ? n : 16));
        if (n) memcpy(bytes.data() + off, p, n);
        return off;
    }
};

// Systolic pair schedule for a team of W warps (see SchedDev): every block
// pair holding at least one listed pair is one group-step.  W = 1: steps are
// matchings (the warp's 4 groups touch disjoint blocks), so the warp can add
// pair forces straight into per-atom forces.  Off-diagonal block pairs are
// packed 4 to a step in the order of a round-robin tournament (circle
// method), diagonal blocks fill free groups of those steps (8 rounds, half
// coefficients: each pair is met twice), and the remaining diagonal blocks
// go 4 to a half step of 4 rounds (rounds 1-3 meet each pair once, round 4
// twice at half coefficients).  W > 1: block pairs dealt round-robin to the
// 4W groups, each with its own partial forces; each warp runs as many steps
// as its busiest group.
struct SchedHost {
    std::vector<uint32_t> ctrl;
    std::vector<float4> rec;
    std::vector<uint32_t> gmask;  // per block: bit q set when group q's partial row holds forces of its atoms
    int base[8] = {0}, steps[8] = {0};
    double listed = 0;  // pair slots weighted by how often a step meets them; must equal the pair count
};

SchedHost build_sched(int n, int W, const std::vector<int> &pidx, const std::vector<float4> &pc) {
    const int nb = (n + 7) / 8, NG = 4 * W;
    auto nonempty = [&](int A, int B) {
        for (int a = 8 * A; a < 8 * A + 8 && a < n; ++a)
            for (int b = (A == B ? a + 1 : 8 * B); b < 8 * B + 8 && b < n; ++b)
                if (pidx[(size_t)a * n + b] >= 0) return true;
        return false;
    };
    std::vector<std::pair<int, int>> bps;
    std::vector<std::vector<int>> glist(NG);  // per group: block-pair index per step, -1 idle
    std::vector<char> half;                   // W = 1: per step, a half (diagonal) step
    if (W == 1) {
        // off-diagonal pairs in circle-method order
        const int ne = nb + (nb & 1);
        for (int rr = 0; rr < ne - 1; ++rr) {
            std::vector<int> arr(ne);
            arr[0] = ne - 1;
            for (int i = 1; i < ne; ++i) arr[i] = (rr + i - 1) % (ne - 1);
            for (int i = 0; i < ne / 2; ++i) {
                int a = arr[i], b = arr[ne - 1 - i];
                if (a > b) std::swap(a, b);
                if (b < nb && nonempty(a, b)) bps.push_back({a, b});
            }
        }
        const size_t n_off = bps.size();
        std::vector<int> diag;
        for (int d = 0; d < nb; ++d)
            if (nonempty(d, d)) diag.push_back(d);
        std::vector<char> done(n_off, 0), dused(diag.size(), 0);
        size_t left = n_off;
        while (left) {
            std::vector<char> used(nb, 0);
            int q = 0;
            for (size_t i = 0; i < n_off && q < 4; ++i) {
                if (done[i] || used[bps[i].first] || used[bps[i].second]) continue;
                used[bps[i].first] = used[bps[i].second] = 1;
                done[i] = 1;
                --left;
                glist[q++].push_back((int)i);
            }
            for (size_t k = 0; k < diag.size() && q < 4; ++k) {  // free groups take diagonal blocks
                if (dused[k] || used[diag[k]]) continue;
                used[diag[k]] = 1;
                dused[k] = 1;
                bps.push_back({diag[k], diag[k]});
                glist[q++].push_back((int)bps.size() - 1);
            }
            for (; q < 4; ++q) glist[q].push_back(-1);
            half.push_back(0);
        }
        int q = 0;
        for (size_t k = 0; k < diag.size(); ++k) {
            if (dused[k]) continue;
            bps.push_back({diag[k], diag[k]});
            glist[q++].push_back((int)bps.size() - 1);
            if (q == 4) {
                half.push_back(1);
                q = 0;
            }
        }
        if (q) {
            for (; q < 4; ++q) glist[q].push_back(-1);
            half.push_back(1);
        }
    } else {
        for (int A = 0; A < nb; ++A)
            for (int B = A; B < nb; ++B)
                if (nonempty(A, B)) bps.push_back({A, B});
        for (size_t i = 0; i < bps.size(); ++i) glist[i % NG].push_back((int)i);
    }
    SchedHost S;
    int off = 0;
    for (int w = 0; w < 8; ++w) {
        int R = 0;
        if (w < W)
            for (int q = 0; q < 4; ++q) R = std::max(R, (int)glist[4 * w + q].size());
        S.base[w] = off;
        S.steps[w] = R;
        off += R;
    }
    const size_t ns = (size_t)std::max(off, 1);
    S.gmask.assign((size_t)std::max(nb, 1), 0u);
    S.ctrl.assign(ns * 4, 0u);
    S.rec.assign(ns * 256, make_float4(0.f, 0.f, 0.f, 0.f));
    for (int w = 0; w < W; ++w)
        for (int q = 0; q < 4; ++q) {
            int st = S.base[w];
            for (size_t k = 0; k < glist[4 * w + q].size(); ++k, ++st) {
                const bool hs = W == 1 && half[k];
                const int bi = glist[4 * w + q][k];
                if (bi < 0) {  // idle: valid flag clear, zero records
                    S.ctrl[4 * (size_t)st + q] = hs ? SCH_HALF : 0u;
                    continue;
                }
                const int A = bps[bi].first, B = bps[bi].second;
                const bool diag = A == B;
                S.gmask[A] |= 1u << (4 * w + q);
                S.gmask[B] |= 1u << (4 * w + q);
                S.ctrl[4 * (size_t)st + q] = (uint32_t)A | ((uint32_t)B << 5) | SCH_VALID | (hs ? SCH_HALF : 0u);
                for (int d = hs ? 1 : 0; d < (hs ? 5 : 8); ++d)
                    for (int sl = 0; sl < 8; ++sl) {
                        const int a = 8 * A + sl, b = 8 * B + ((sl + d) & 7);
                        if (a >= n || b >= n || a == b) continue;
                        const int i = std::min(a, b), j = std::max(a, b);
                        const int pp = pidx[(size_t)i * n + j];
                        if (pp < 0) continue;
                        const size_t o = 256 * (size_t)st + 32 * d + 8 * q + sl;
                        float4 c = pc[pp];
                        // met twice in the step: half each time (exact in FP32)
                        const bool twice = diag && (!hs || d == 4);
                        if (twice) {
                            c.x *= 0.5f; c.y *= 0.5f; c.z *= 0.5f; c.w *= 0.5f;
                        }
                        S.rec[o] = c;
                        S.listed += twice ? 0.5 : 1.0;
                    }
            }
        }
    // by round pair for the paired FP32 rounds: rounds (2p, 2p + 1), or (2p +
    // 1, 2p + 2) in a half step
    std::vector<float4> by_round = std::move(S.rec);
    S.rec.assign(ns * 256, make_float4(0.f, 0.f, 0.f, 0.f));
    for (size_t st = 0; st < ns; ++st) {
        const bool hs = (S.ctrl[4 * st] & SCH_HALF) != 0;
        for (int p = 0; p < (hs ? 2 : 4); ++p) {
            const int d0 = hs ? 2 * p + 1 : 2 * p;
            for (int lane = 0; lane < 32; ++lane) {
                const float4 c0 = by_round[256 * st + 32 * d0 + lane], c1 = by_round[256 * st + 32 * (d0 + 1) + lane];
                S.rec[256 * st + 64 * p + lane] = make_float4(c0.x, c1.x, c0.y, c1.y);
                S.rec[256 * st + 64 * p + 32 + lane] = make_float4(c0.z, c1.z, c0.w, c1.w);
            }
        }
    }
    return S;
}

}  // namespace

extern "C" int load_ligand(dock_ctx *ctx, int n, const double *xyz, const int *type, const double *charge, int nb,
                           const int *bonds, const int *rot, dock_ligand **out) {
    if (!ctx || !out) return DOCK_ERR_INVALID;
    *out = nullptr;
    if (n < 1 || n > DOCK_MAX_ATOMS) return set_err(ctx, DOCK_ERR_SIZE, "atom count must be 1..255");
    if (!xyz || !type || !charge || nb < 0 || (nb > 0 && (!bonds || !rot)))
        return set_err(ctx, DOCK_ERR_INVALID, "null ligand array");
    for (int i = 0; i < n; ++i) {
        if (type[i] < 0 || type[i] >= DOCK_NTYPES) return set_err(ctx, DOCK_ERR_TYPE, "unknown atom type");
        if (!isfinite(xyz[3 * i]) || !isfinite(xyz[3 * i + 1]) || !isfinite(xyz[3 * i + 2]) || !isfinite(charge[i]))
            return set_err(ctx, DOCK_ERR_INVALID, "non-finite coordinate or charge");
    }
    int nt = 0;
    std::vector<std::vector<std::pair<int, int>>> adj(n);  // (neighbour, bond)
    for (int b = 0; b < nb; ++b) {
        const int u = bonds[2 * b], v = bonds[2 * b + 1];
        if (u < 0 || v < 0 || u >= n || v >= n || u == v) return set_err(ctx, DOCK_ERR_INVALID, "bad bond");
        adj[u].push_back({v, b});
        adj[v].push_back({u, b});
        nt += rot[b] ? 1 : 0;
    }
    if (nt > DOCK_MAX_TORSIONS) return set_err(ctx, DOCK_ERR_SIZE, "more than 32 rotatable bonds");
    // flood fill from `start`, skipping bond `skip` (and rotatable bonds if rigid)
    auto flood = [&](int start, int skip, bool rigid, std::vector<int> &lab, int id) {
        std::vector<int> st{start};
        lab[start] = id;
        int cnt = 0;
        while (!st.empty()) {
            const int a = st.back();
            st.pop_back();
            ++cnt;
            for (auto [w, b] : adj[a])
                if (b != skip && !(rigid && rot[b]) && lab[w] < 0) {
                    lab[w] = id;
                    st.push_back(w);
                }
        }
        return cnt;
    };
    std::vector<int> lab(n, -1);
    if (flood(0, -1, false, lab, 0) != n) return set_err(ctx, DOCK_ERR_DISCONNECTED, "bond graph is not connected");
    for (int b = 0; b < nb; ++b) {
        if (!rot[b]) continue;
        std::fill(lab.begin(), lab.end(), -1);
        flood(bonds[2 * b], b, false, lab, 0);
        if (lab[bonds[2 * b + 1]] >= 0) return set_err(ctx, DOCK_ERR_RING, "rotatable bond inside a ring");
    }
    // rigid fragments, numbered by their lowest atom
    std::vector<int> comp(n, -1), fsize;
    for (int i = 0; i < n; ++i)
        if (comp[i] < 0) fsize.push_back(flood(i, -1, true, comp, (int)fsize.size()));
    const int F = (int)fsize.size();
    int root = 0;
    for (int f = 1; f < F; ++f)
        if (fsize[f] > fsize[root]) root = f;
    // torsion tree: depth-first preorder of fragments from the root; children
    // in the order of their entering bond in the input
    std::vector<int> rank(nb, -1);
    for (int b = 0, k = 0; b < nb; ++b)
        if (rot[b]) rank[b] = k++;
    std::vector<std::vector<std::pair<int, int>>> fadj(F);  // (fragment, bond)
    for (int b = 0; b < nb; ++b)
        if (rot[b]) {
            fadj[comp[bonds[2 * b]]].push_back({comp[bonds[2 * b + 1]], b});
            fadj[comp[bonds[2 * b + 1]]].push_back({comp[bonds[2 * b]], b});
        }
    std::vector<int> order, fparent(F, -1), fbond(F, -1), newf(F, -1);
    {
        std::vector<std::pair<int, int>> st{{root, -1}};
        std::vector<char> vis(F, 0);
        while (!st.empty()) {
            auto [f, via] = st.back();
            st.pop_back();
            if (vis[f]) continue;
            vis[f] = 1;
            fbond[f] = via;
            newf[f] = (int)order.size();
            order.push_back(f);
            std::vector<std::pair<int, int>> kids;
            for (auto [g, b] : fadj[f])
                if (!vis[g]) kids.push_back({b, g});
            std::sort(kids.begin(), kids.end());
            for (auto it = kids.rbegin(); it != kids.rend(); ++it) {
                fparent[it->second] = f;
                st.push_back({it->second, it->first});
            }
        }
    }
    if ((int)order.size() != F) return set_err(ctx, DOCK_ERR_DISCONNECTED, "torsion tree is not connected");
    std::vector<int> depth(F, 0), sub_end(F, 0);
    for (int k = 1; k < F; ++k) depth[k] = depth[newf[fparent[order[k]]]] + 1;
    for (int k = F - 1; k >= 0; --k) {
        int e = k + 1;
        for (int j = k + 1; j < F && depth[j] > depth[k]; ++j) e = j + 1;
        sub_end[k] = e;
    }
    // atoms: fragment by fragment in preorder, ascending input index inside
    std::vector<int> perm, inv(n, -1);
    std::vector<int4> frag(F);
    for (int k = 0; k < F; ++k) {
        const int f = order[k], begin = (int)perm.size();
        for (int i = 0; i < n; ++i)
            if (comp[i] == f) {
                inv[i] = (int)perm.size();
                perm.push_back(i);
            }
        frag[k] = make_int4(begin, (int)perm.size(), k ? newf[fparent[f]] : -1, depth[k]);
    }
    double c[3] = {0, 0, 0};
    for (int i = 0; i < n; ++i)
        for (int a = 0; a < 3; ++a) c[a] += xyz[3 * i + a];
    for (int a = 0; a < 3; ++a) c[a] /= n;
    std::vector<double> ref64(3 * n), q64(n);
    std::vector<float4> ref(n);
    std::vector<int> meta(n), types(n);
    for (int k = 0; k < n; ++k) {
        const int i = perm[k];
        for (int a = 0; a < 3; ++a) ref64[3 * k + a] = xyz[3 * i + a] - c[a];
        q64[k] = charge[i];
        ref[k] = make_float4((float)ref64[3 * k], (float)ref64[3 * k + 1], (float)ref64[3 * k + 2], (float)charge[i]);
        meta[k] = type[i] | (comp[i] >= 0 ? newf[comp[i]] << 8 : 0);
        types[k] = type[i];
    }
    const int T = F - 1;
    std::vector<float4> tu(std::max(T, 1)), tb(std::max(T, 1));
    std::vector<int2> tab(std::max(T, 1));
    std::vector<int> tgene(std::max(T, 1)), fdepth_max(1, 0);
    int max_depth = 0;
    for (int k = 0; k < T; ++k) {
        const int f = order[k + 1], b = fbond[f];
        int ua = bonds[2 * b], ub = bonds[2 * b + 1];
        if (comp[ub] != f) std::swap(ua, ub);  // ub on the child (moving) side
        const int ia = inv[ua], ib = inv[ub];
        double u[3] = {ref64[3 * ib] - ref64[3 * ia], ref64[3 * ib + 1] - ref64[3 * ia + 1],
                       ref64[3 * ib + 2] - ref64[3 * ia + 2]};
        const double len = sqrt(u[0] * u[0] + u[1] * u[1] + u[2] * u[2]);
        if (!(len > 0)) return set_err(ctx, DOCK_ERR_INVALID, "zero-length rotatable bond");
        tu[k] = make_float4((float)(u[0] / len), (float)(u[1] / len), (float)(u[2] / len), 0.f);
        tb[k] = make_float4((float)ref64[3 * ib], (float)ref64[3 * ib + 1], (float)ref64[3 * ib + 2], 0.f);
        tab[k] = make_int2(ia, ib);
        tgene[k] = 7 + rank[b];
        max_depth = std::max(max_depth, depth[k + 1]);
    }
    // bond-graph distances (input numbering)
    std::vector<int> dist((size_t)n * n, -1);
    for (int s0 = 0; s0 < n; ++s0) {
        int *d = dist.data() + (size_t)s0 * n;
        std::queue<int> q;
        d[s0] = 0;
        q.push(s0);
        while (!q.empty()) {
            const int a = q.front();
            q.pop();
            for (auto [w, b] : adj[a])
                if (d[w] < 0) {
                    d[w] = d[a] + 1;
                    q.push(w);
                }
        }
    }
    // pair list: different rigid fragments, >= 4 bonds apart
    std::vector<uint32_t> pij;
    std::vector<float4> pc;
    std::vector<double> pc64;
    for (int i = 0; i < n; ++i)
        for (int j = i + 1; j < n; ++j) {
            const int I = perm[i], J = perm[j];
            if (comp[I] == comp[J] || dist[(size_t)I * n + J] < 4) continue;
            double c12, c6, c10;
            ff::vdw_coefs(type[I], type[J], c12, c6, c10);
            const double qq = ff::kWel * ff::kCoulomb * charge[I] * charge[J];
            const double ds = ff::kWds * (ff::solv(type[I], charge[I]) * ff::kTypes[type[J]].vol +
                                          ff::solv(type[J], charge[J]) * ff::kTypes[type[I]].vol);
            pij.push_back((uint32_t)i | ((uint32_t)j << 16));
            // c6 and c10 are never both non-zero: the sign of cn selects the exponent
            pc.push_back(make_float4((float)c12, c10 != 0.0 ? -(float)c10 : (float)c6, (float)qq, (float)ds));
            pc64.insert(pc64.end(), {c12, c6, c10, qq, ds});
        }
    const int P = (int)pij.size();
    std::vector<int> pidx((size_t)n * n, -1);
    for (int p = 0; p < P; ++p) pidx[(size_t)(pij[p] & 0xffff) * n + (pij[p] >> 16)] = p;
    SchedHost sched[4];
    for (int k = 0; k < 4; ++k) {
        sched[k] = build_sched(n, 1 << k, pidx, pc);
        if (sched[k].listed != (double)P) return set_err(ctx, DOCK_ERR_INVALID, "internal error: pair schedule incomplete");
    }
    std::vector<std::vector<uint32_t>> lists(n);
    for (int p = 0; p < P; ++p) {
        const int i = pij[p] & 0xffff, j = pij[p] >> 16;
        lists[i].push_back((uint32_t)p | ((uint32_t)j << 16));
        lists[j].push_back((uint32_t)p | ((uint32_t)i << 16));
    }
    std::vector<int> adj_off(n + 1, 0);
    std::vector<uint32_t> adjv;
    for (int i = 0; i < n; ++i) {
        adj_off[i] = (int)adjv.size();
        adjv.insert(adjv.end(), lists[i].begin(), lists[i].end());
    }
    adj_off[n] = (int)adjv.size();

    Blob B;
    const size_t o_ref = B.add(ref.data(), n * sizeof(float4));
    const size_t o_meta = B.add(meta.data(), n * sizeof(int));
    const size_t o_perm = B.add(perm.data(), n * sizeof(int));
    const size_t o_frag = B.add(frag.data(), F * sizeof(int4));
    const size_t o_sub = B.add(sub_end.data(), F * sizeof(int));
    const size_t o_tu = B.add(tu.data(), T * sizeof(float4));
    const size_t o_tb = B.add(tb.data(), T * sizeof(float4));
    const size_t o_tab = B.add(tab.data(), T * sizeof(int2));
    const size_t o_tg = B.add(tgene.data(), T * sizeof(int));
    std::vector<int2> trange(std::max(T, 1));
    for (int k = 0; k < T; ++k) trange[k] = make_int2(frag[k + 1].x, frag[sub_end[k + 1] - 1].y);
    const size_t o_trg = B.add(trange.data(), T * sizeof(int2));
    const size_t o_pij = B.add(pij.data(), P * sizeof(uint32_t));
    const size_t o_pc = B.add(pc.data(), P * sizeof(float4));
    const size_t o_aoff = B.add(adj_off.data(), (n + 1) * sizeof(int));
    const size_t o_adj = B.add(adjv.data(), adjv.size() * sizeof(uint32_t));
    const size_t o_r64 = B.add(ref64.data(), 3 * n * sizeof(double));
    const size_t o_pc64 = B.add(pc64.data(), pc64.size() * sizeof(double));
    const size_t o_q64 = B.add(q64.data(), n * sizeof(double));
    size_t o_sc[4], o_sr[4], o_sm[4];
    for (int k = 0; k < 4; ++k) {
        o_sc[k] = B.add(sched[k].ctrl.data(), sched[k].ctrl.size() * sizeof(uint32_t));
        o_sr[k] = B.add(sched[k].rec.data(), sched[k].rec.size() * sizeof(float4));
        o_sm[k] = B.add(sched[k].gmask.data(), sched[k].gmask.size() * sizeof(uint32_t));
    }

    dock_ligand *L = new dock_ligand();
    L->blob_bytes = B.bytes.size();
    L->blob = dev_alloc(ctx, L->blob_bytes, nullptr);
    if (!L->blob) {
        delete L;
        return set_err(ctx, DOCK_ERR_OOM, "ligand allocation failed");
    }
    cudaError_t e = cudaMemcpyAsync(L->blob, B.bytes.data(), L->blob_bytes, cudaMemcpyHostToDevice, nullptr);
    if (!e) e = cudaStreamSynchronize(nullptr);
    if (e) {
        dev_free(ctx, L->blob, nullptr);
        delete L;
        return cuda_err(ctx, e, "ligand upload");
    }
    const unsigned char *base = (const unsigned char *)L->blob;
    LigandDev &d = L->dev;
    d.n_atoms = n;
    d.n_tors = T;
    d.n_frag = F;
    d.n_pairs = P;
    d.n_genes = 7 + T;
    d.max_depth = max_depth;
    d.ref = (const float4 *)(base + o_ref);
    d.meta = (const int *)(base + o_meta);
    d.perm = (const int *)(base + o_perm);
    d.frag = (const int4 *)(base + o_frag);
    d.sub_end = (const int *)(base + o_sub);
    d.tors_u = (const float4 *)(base + o_tu);
    d.tors_b = (const float4 *)(base + o_tb);
    d.tors_ab = (const int2 *)(base + o_tab);
    d.tors_gene = (const int *)(base + o_tg);
    d.tors_range = (const int2 *)(base + o_trg);
    d.pair_ij = (const uint32_t *)(base + o_pij);
    d.pair_c = (const float4 *)(base + o_pc);
    d.adj_off = (const int *)(base + o_aoff);
    d.adj = (const uint32_t *)(base + o_adj);
    d.ref64 = (const double *)(base + o_r64);
    d.pair_c64 = (const double *)(base + o_pc64);
    d.q64 = (const double *)(base + o_q64);
    d.nb8 = (n + 7) & ~7;
    for (int k = 0; k < 4; ++k) {
        d.sched[k].ctrl = (const uint32_t *)(base + o_sc[k]);
        d.sched[k].rec = (const float4 *)(base + o_sr[k]);
        d.sched[k].gmask = (const uint32_t *)(base + o_sm[k]);
        for (int w = 0; w < 8; ++w) {
            d.sched[k].base[w] = sched[k].base[w];
            d.sched[k].steps[w] = sched[k].steps[w];
        }
    }
    L->types = types;
    *out = L;
    return DOCK_OK;
}

extern "C" {

int ligand_info(const dock_ligand *l, int *n_atoms, int *n_torsions, int *n_genes, int *n_pairs, int *n_fragments) {
    if (!l) return DOCK_ERR_INVALID;
    if (n_atoms) *n_atoms = l->dev.n_atoms;
    if (n_torsions) *n_torsions = l->dev.n_tors;
    if (n_genes) *n_genes = l->dev.n_genes;
    if (n_pairs) *n_pairs = l->dev.n_pairs;
    if (n_fragments) *n_fragments = l->dev.n_frag;
    return DOCK_OK;
}

int ligand_device_bytes(const dock_ligand *l, size_t *bytes) {
    if (!l || !bytes) return DOCK_ERR_INVALID;
    *bytes = l->blob_bytes;
    return DOCK_OK;
}

int free_ligand(dock_ctx *ctx, dock_ligand *l) {
    if (!ctx || !l) return DOCK_ERR_INVALID;
    cudaStreamSynchronize(nullptr);
    dev_free(ctx, l->blob, nullptr);
    delete l;
    return DOCK_OK;
}

// ---------------------------------------------------------------------------
// batched evaluation

static int score_common(dock_ctx *ctx, const dock_grids *g, const dock_ligand *l, const float *geno, int B, float *E,
                        float *grad, void *stream) {
    if (!ctx) return DOCK_ERR_INVALID;
    if (!g || !l || B < 0 || (B > 0 && (!geno || !E))) return set_err(ctx, DOCK_ERR_INVALID, "invalid argument");
    int rc = check_maps(ctx, g, l);
    if (rc) return rc;
    if (B == 0) return DOCK_OK;
    const EvalLayout W = eval_layout(l->dev.n_atoms, l->dev.n_frag, l->dev.nb8, grad != nullptr, 1);
    if (!evaluator_smem_ok(ctx, W, 1)) return set_err(ctx, DOCK_ERR_SIZE, "ligand too large for shared memory");
    cudaError_t e = launch_score(ctx, l->dev, g->dev, geno, B, E, grad, (cudaStream_t)stream);
    return e ? cuda_err(ctx, e, "score kernel") : DOCK_OK;
}

int score_batch(dock_ctx *ctx, const dock_grids *g, const dock_ligand *l, const float *geno, int B, float *E,
                void *stream) {
    return score_common(ctx, g, l, geno, B, E, nullptr, stream);
}

int score_grad_batch(dock_ctx *ctx, const dock_grids *g, const dock_ligand *l, const float *geno, int B, float *E,
                     float *grad, void *stream) {
    if (ctx && B > 0 && !grad) return set_err(ctx, DOCK_ERR_INVALID, "null gradient buffer");
    return score_common(ctx, g, l, geno, B, E, grad, stream);
}

int pose_batch(dock_ctx *ctx, const dock_ligand *l, const float *geno, int B, float *xyz, void *stream) {
    if (!ctx) return DOCK_ERR_INVALID;
    if (!l || B < 0 || (B > 0 && (!geno || !xyz))) return set_err(ctx, DOCK_ERR_INVALID, "invalid argument");
    if (B == 0) return DOCK_OK;
    const EvalLayout W = eval_layout(l->dev.n_atoms, l->dev.n_frag, l->dev.nb8, false, 1);
    if (!evaluator_smem_ok(ctx, W, 1)) return set_err(ctx, DOCK_ERR_SIZE, "ligand too large for shared memory");
    cudaError_t e = launch_pose(ctx, l->dev, geno, B, xyz, (cudaStream_t)stream);
    return e ? cuda_err(ctx, e, "pose kernel") : DOCK_OK;
}

}  // extern "C"
