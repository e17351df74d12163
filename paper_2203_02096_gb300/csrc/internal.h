// internal.h -- device data layouts and launch helpers of libdock.so.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "dock.h"

#define DOCK_WARP 32

// Ligand on the device.  Atoms are renumbered so that each rigid fragment is
// a contiguous range and fragments follow a depth-first preorder of the
// torsion tree (fragment 0 = root); then the atoms moved by the torsion
// entering fragment f are exactly the fragments [f, sub_end[f]).  Internal
// torsion k is the bond entering fragment k+1.
// Systolic pair schedule for a team of W warps (4W groups of 8 lanes).
// Atoms form blocks of 8; a step is one block pair (A, B), 8 rounds: in
// round d lane l of the group pairs atom 8A + l with atom 8B + (l + d) mod 8.
// A diagonal step (A == B) meets every pair of its block twice (rounds d and
// 8 - d), each time with half the coefficients; a half step (one-warp teams,
// every group diagonal) runs rounds 1-4 only, round 4 at half coefficients.
// ctrl[step][group of the warp] packs A, B, a valid flag and the half-step
// flag (set on all four groups of a half step).  Pair coefficients (c12, cn,
// qq, ds) -- cn = c6 for 12-6 pairs, -c10 for 12-10 H-bond pairs -- zero for
// pairs outside the pair list, by round pair: rounds (d, d + 1) = (2p, 2p + 1),
// or (2p + 1, 2p + 2) in a half step; rec[step][p][0][lane] = (c12, c12', cn,
// cn') and rec[step][p][1][lane] = (qq, qq', ds, ds'), ' = round d + 1.
struct SchedDev {
    const uint32_t *ctrl;
    const float4 *rec;
    const uint32_t *gmask;  // [block] groups whose partial-force rows touch the block (W > 1)
    int base[8];   // first step of warp w
    int steps[8];  // steps of warp w
};

#define SCH_A(c) ((c) & 31u)
#define SCH_B(c) (((c) >> 5) & 31u)
#define SCH_VALID 0x10000u
#define SCH_HALF 0x20000u  // W = 1 half step: diagonal blocks, rounds 1-4 only

struct LigandDev {
    int n_atoms, n_tors, n_frag, n_pairs, n_genes, max_depth;
    int nb8;                  // atoms rounded up to a multiple of 8
    SchedDev sched[4];        // for W = 1, 2, 4, 8
    const float4 *ref;        // [n] centred reference coords, w = partial charge
    const int *meta;          // [n] type | fragment << 8
    const int *perm;          // [n] internal atom -> input atom
    const int4 *frag;         // [F] (atom begin, atom end, parent, depth)
    const int *sub_end;       // [F] end of the fragment's subtree (fragment numbering)
    const int2 *tors_range;   // [T] contiguous atom range [x, y) that torsion k moves
    const float4 *tors_u;     // [T] unit bond axis a->b in the reference frame
    const float4 *tors_b;     // [T] reference position of axis atom b
    const int2 *tors_ab;      // [T] internal atom indices (a, b)
    const int *tors_gene;     // [T] genotype index of internal torsion k
    const uint32_t *pair_ij;  // [P] i | j << 16, internal atom indices
    const float4 *pair_c;     // [P] (c12, cn, w_el * 332.06 * q_i q_j, w_ds (S_i V_j + S_j V_i)), cn as above
    const int *adj_off;       // [n+1] CSR over atoms of the pairs they take part in
    const uint32_t *adj;      // [2P] pair index | partner atom << 16
    const double *ref64;      // [n][3] centred reference coords (FP64 re-score)
    const double *pair_c64;   // [P][5] c12, c6, c10, qq, ds (FP64 re-score)
    const double *q64;        // [n] charges (FP64 re-score)
};

// Receptor grids on the device.  cells: z-column quad copy.  For map m,
// column (ix, iy) (ix < nx-1, iy < ny-1) and node plane iz < nz, the quad
// (v(ix,iy,iz), v(ix+1,iy,iz), v(ix,iy+1,iz), v(ix+1,iy+1,iz)) is float4
// number m*mstride + (iy*(nx-1) + ix)*nz + iz, mstride = (nx-1)(ny-1)nz.
// A cell's 8 corners are two adjacent quads (iz, iz+1): one 32-byte read,
// 4x the node-major size (a full cell-major copy would be 8x).
struct GridDev {
    const float4 *cells;
    long long mstride;        // quads per map
    const float *nodes;       // [M][nz][ny][nx] node-major copy
    const int *map_of_type;   // [8] ligand type -> map, -1 if absent
    int nx, ny, nz, M;
    float ox, oy, oz, h, inv_h;
    int emap, dmap;
    float box_lo[3], box_len[3];  // search box for initial translations (FP32, rounded once)
    double ox64, oy64, oz64, h64;
};

// Shared-memory scratch of one evaluating team, offsets in floats (each a
// multiple of 4 so float4 views are aligned).
struct EvalLayout {
    int geno, grad, red, M, fs, x, z, f, tq, pf, cst, total;
};

__host__ __device__ inline int round4(int v) { return (v + 3) & ~3; }

// W: warps of the team (partials: 4W groups x nb8 atoms).
__host__ __device__ inline EvalLayout eval_layout(int n_atoms, int n_frag, int nb8, bool grad, int W) {
    EvalLayout w;
    int o = 0;
    w.geno = o; o += 48 * W;          // a copy per warp
    w.grad = o; o += 48;
    w.red = o; o += 32;               // team sums: two halves of 8 warp partials, then 8 energy partials
    w.M = o; o += 12 * n_frag * W;    // a copy per warp
    w.fs = o;                         // W = 1: fragment sums live in the staged-cell area (cst)
    w.x = o; o += 4 * nb8;            // positions, pair-major: (x, x', y, y') per atom
    w.z = o; o += 2 * nb8;            // (z, z') per atom
    w.f = o; o += grad ? 4 * nb8 : 0;
    w.tq = o; o += (grad && W > 1) ? 4 * n_atoms : 0;  // W = 1: torques live in cst
    w.pf = o; o += (grad && W > 1) ? 4 * 4 * W * (nb8 + 4) : 0;  // rows nb8 + 4 apart; W = 1 adds straight into f
    w.cst = o; o += 24 * nb8;  // staged map cells: 6 float4 per atom
    w.total = round4(o);
    return w;
}

// Library-side objects behind the opaque handles.
struct TimedLaunch {
    int kernel;
    cudaEvent_t start, stop;
};

struct dock_ctx {
    int device = 0;
    int num_sms = 0;
    size_t smem_optin = 0;
    dock_allocator alloc{};
    bool has_alloc = false;
    std::string err;
    bool timing = false;
    std::vector<TimedLaunch> pending;
    std::vector<cudaEvent_t> event_pool;
    std::vector<std::string> kernel_names;
    std::vector<double> kernel_ms;
    std::vector<int64_t> kernel_launches;
    int64_t launches = 0;
    int *d_flag = nullptr;  // device error word: 0 = fine
    long long *h_status = nullptr;  // pinned host words read back by the Solis-Wets docking loop
    int score_min_blocks = 1;       // register cap of the batched scorers (DOCK_OPT_SCORE_BLOCKS)
    int batch_min_blocks = 4;       // register cap of the persistent docking kernel (DOCK_OPT_BATCH_BLOCKS)
};

struct dock_grids {
    GridDev dev{};
    int map_of_type[8] = {-1, -1, -1, -1, -1, -1, -1, -1};
    void *cells_mem = nullptr;
    void *nodes_mem = nullptr;
    void *lut_mem = nullptr;
    int n_maps = 0;
    std::vector<int> map_type;
};

struct dock_ligand {
    LigandDev dev{};
    void *blob = nullptr;
    size_t blob_bytes = 0;
    std::vector<int> types;  // input types, for the map check
};

// ---- helpers shared by the library's translation units (host side) ----
int set_err(dock_ctx *ctx, int code, const std::string &msg);
int cuda_err(dock_ctx *ctx, cudaError_t e, const char *what);
void *dev_alloc(dock_ctx *ctx, size_t bytes, cudaStream_t s);
void dev_free(dock_ctx *ctx, void *p, cudaStream_t s);
int kernel_id(dock_ctx *ctx, const char *name);
long long *host_status(dock_ctx *ctx);
int check_sw(dock_ctx *ctx, const dock_params &p);  // ls_method and Solis-Wets constants
int tune_batch_launch(dock_ctx *ctx, const dock_grids *grids, const dock_ligand *const *ligs, int n_ligs,
                      const dock_params &P, int wpb, int min_blocks, int reps, double *ms);  // 2 pinned words, allocated on first use; NULL on failure
void timing_begin(dock_ctx *ctx, int kid, cudaStream_t s, TimedLaunch *tl);
void timing_end(dock_ctx *ctx, cudaStream_t s, TimedLaunch *tl);
int check_maps(dock_ctx *ctx, const dock_grids *g, const dock_ligand *l);
int evaluator_smem_ok(dock_ctx *ctx, const EvalLayout &w, int warps);

// Kernel launchers (defined in the .cu files).
cudaError_t launch_relayout(const GridDev &g, float4 *cells, cudaStream_t s);
cudaError_t launch_build_maps(int n_rec, const float4 *rec_rel, const int *rtype, int nx, int ny, int nz, double h,
                              int n_tmaps, const int *map_types, float *nodes, cudaStream_t s);
cudaError_t launch_rescore64(dock_ctx *ctx, const LigandDev &L, const GridDev &G, const float *geno, int B, double *E,
                             cudaStream_t s);
cudaError_t launch_score(dock_ctx *ctx, const LigandDev &L, const GridDev &G, const float *geno, int B, float *E,
                         float *grad, cudaStream_t s);
cudaError_t launch_pose(dock_ctx *ctx, const LigandDev &L, const float *geno, int B, float *xyz, cudaStream_t s);
// Looks up the no-allocation scratch array on the current device (search.cu).
int noalloc_prepare(dock_ctx *ctx);

