/*
 * dock.h -- C ABI of the GB300 docking library (libdock.so, CUDA sm_103a).
 *
 * The library evaluates and optimises ligand poses against receptor grids:
 * the population-parallel pose evaluation inside a Lamarckian genetic search
 * (paper, Section II-A).  A genotype is
 *     [ t_x, t_y, t_z,  q_w, q_x, q_y, q_z,  tau_0 ... tau_{T-1} ]   (FP32)
 * G = 7 + T genes: translation of the ligand centroid (A), an orientation
 * quaternion (any non-zero norm; normalised on use), and one torsion angle
 * (radians, relative to the input conformation) per rotatable bond, in the
 * order the rotatable bonds appear in the bond list given to load_ligand.
 *
 * Conventions for every entry point:
 *   - return 0 (DOCK_OK) or a negative DOCK_ERR_* code; nothing aborts the
 *     process; dock_last_error(ctx) gives a one-line description;
 *   - "host" pointers are read or written before the call returns;
 *   - "device" pointers are CUDA device memory owned by the caller, used in
 *     stream order on the given stream (cudaStream_t passed as void*, NULL =
 *     the legacy default stream); the call returns once the work is queued;
 *   - handles (dock_ctx, dock_grids, dock_ligand) are owned by the library
 *     and released by the matching free call; a handle is used by one host
 *     thread at a time.
 * All arithmetic on the device is FP32, except the FP64 re-scoring of each
 * run's best pose in dock()/dock_async().
 */
#ifndef GB300_DOCK_H
#define GB300_DOCK_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define DOCK_OK 0
#define DOCK_ERR_INVALID (-1)      /* bad argument (null, size, range)             */
#define DOCK_ERR_CUDA (-2)         /* a CUDA runtime call failed                   */
#define DOCK_ERR_OOM (-3)          /* device allocation failed                     */
#define DOCK_ERR_DISCONNECTED (-4) /* ligand bond graph is not connected           */
#define DOCK_ERR_RING (-5)         /* a rotatable bond lies in a ring              */
#define DOCK_ERR_SIZE (-6)         /* too many atoms (>255) or torsions (>32)      */
#define DOCK_ERR_TYPE (-7)         /* unknown atom type code                       */
#define DOCK_ERR_NOMAP (-8)        /* a ligand atom type has no map in the grids   */
#define DOCK_ERR_DEVICE (-9)       /* a kernel reported an error through its flag  */
#define DOCK_ERR_BUSY (-10)        /* the serving queue has no free slot right now */

#define DOCK_MAX_ATOMS 255
#define DOCK_MAX_TORSIONS 32

/* Atom type codes (ligand and receptor): C, A (aromatic C), N, NA (acceptor
 * N), OA (acceptor O), SA (acceptor S), HD (donor H). */
enum { DOCK_C = 0, DOCK_A = 1, DOCK_N = 2, DOCK_NA = 3, DOCK_OA = 4, DOCK_SA = 5, DOCK_HD = 6, DOCK_NTYPES = 7 };
/* map_type codes for the two charge maps in load_grids */
#define DOCK_MAP_ELEC (-1)
#define DOCK_MAP_DESOLV (-2)

typedef struct dock_ctx dock_ctx;
typedef struct dock_grids dock_grids;
typedef struct dock_ligand dock_ligand;

/* Optional device allocator.  alloc returns device memory of >= bytes,
 * 256-byte aligned, usable on `stream`, or NULL; free releases it.  With no
 * allocator the library uses cudaMalloc / cudaFree. */
typedef struct {
    void *(*alloc)(size_t bytes, void *stream, void *user);
    void (*free)(void *ptr, void *stream, void *user);
    void *user;
} dock_allocator;

/* Search parameters (paper, Section II-A: population 150, crossover,
 * fitness-based selection, local search on a random sample of each
 * generation; the rates and the ADADELTA and Solis-Wets constants are this
 * library's).  Local search: ADADELTA (default; one score+gradient per
 * iteration, ls_iters iterations) or Solis-Wets (the paper's miniapp search,
 * Solis and Wets 1981: adaptive random steps with a bias term, energies
 * only, one or two per iteration, at most ls_iters <= 6553 iterations, ends
 * early once the step scale falls below sw_rho_lo).  Evaluations are
 * counted as computed; a run stops at the first generation boundary where
 * its count reaches max_evals. */
typedef struct {
    int pop_size;      /* individuals per run (>= 2), default 150                  */
    int nruns;         /* independent runs, default 10                              */
    int64_t max_evals; /* per-run evaluation budget, default 100000                 */
    int ls_count;      /* local searches per generation; default ceil(6% pop_size)  */
    int ls_iters;      /* iterations per local search, default 100                  */
    float rho, eps;    /* ADADELTA decay and conditioner, default 0.8, 1e-2         */
    float p_tour;      /* probability the fitter of two wins a tournament, 0.6      */
    float p_cross;     /* two-point crossover probability, 0.8                      */
    float p_mut;       /* per-gene-block mutation probability, 0.02                 */
    float trans_mut;   /* translation mutation half-width (A), 2.0                  */
    int ls_threads;    /* threads evaluating one local-search chain: 32, 64, 128,
                          256, or 0 = chosen from the chain count (the paper's
                          threads-per-block knob, Section V-B); default 0       */
    int ls_method;     /* 0 = ADADELTA (default), 1 = Solis-Wets                    */
    float sw_rho0;     /* Solis-Wets step scale at the start, default 1.0           */
    float sw_rho_lo;   /* ... the search ends once it is below this, default 0.01   */
    float sw_expand;   /* scale factor after sw_succ successes in a row, 2.0        */
    float sw_contract; /* scale factor after sw_fail failures in a row, 0.5         */
    int sw_succ, sw_fail; /* default 4, 4                                          */
    float sw_step[3];  /* deviation half-widths at scale 1: translation (A) 1.0,
                          quaternion component 0.2, torsion (rad) 0.75             */
    int batch_warps;   /* warps per block of dock_batch's persistent kernel: 1, 2,
                          4, or 0 = as many (<= 4) as shared memory allows;
                          results do not depend on it; default 0                */
    int batch_pack;    /* dock_batch packing: 0 = one launch over all tasks,
                          largest ligands first (default); 1 = by atom count:
                          ligands in classes of up to 32, 64, 96, 128 and 255
                          atoms, one launch per class (largest class first),
                          each sizing its shared memory, hence its warps per
                          SM, for its own largest ligand; results do not
                          depend on it                                          */
} dock_params;

/* Library version (major*10000 + minor*100 + patch). */
int dock_version(void);

/* Fills *p with the defaults listed in dock_params. */
void dock_default_params(dock_params *p);

/* Creates a context on CUDA device `device`.  alloc may be NULL. */
int dock_create(dock_ctx **out, int device, const dock_allocator *alloc);
/* Releases the context; grids and ligands must be freed first. */
int dock_destroy(dock_ctx *ctx);
/* One-line description of the last error on this context ("" if none). */
const char *dock_last_error(const dock_ctx *ctx);

/* ---- receptor grids: the "reaction field for the protein" (Section II-A) ----
 * maps: host, [n_maps][dims[2]][dims[1]][dims[0]] FP32, x fastest; node
 * (i,j,k) sits at origin + (i,j,k)*spacing.  map_type[m] is the ligand atom
 * type served by map m, or DOCK_MAP_ELEC (potential per unit ligand charge)
 * or DOCK_MAP_DESOLV (desolvation per unit |charge|); exactly one of each.
 * An atom of type t and charge q at x scores M_t(x) + q E(x) + |q| D(x),
 * read by trilinear interpolation; outside the box the read is clamped and
 * 10 kcal/mol/A^2 times the squared distance outside is added per axis.
 * The library keeps its own device copy.  Errors: dims < 2, spacing <= 0,
 * non-finite values, duplicate or missing charge maps, OOM. */
int load_grids(dock_ctx *ctx, const float *maps, int n_maps, const int dims[3], const double origin[3],
               double spacing, const int *map_type, dock_grids **out);

/* Builds the maps on the device from receptor atoms (host arrays: xyz
 * [n_rec][3] A, type codes, partial charges), for ligand types
 * map_types[0..n_type_maps), plus the electrostatic and desolvation maps:
 * the direct sum over all receptor atoms of the same pair terms the ligand
 * uses internally (no cutoff), type maps capped at +1e5 kcal/mol. */
int build_grids(dock_ctx *ctx, int n_rec, const double *rxyz, const int *rtype, const double *rq,
                const int dims[3], const double origin[3], double spacing, int n_type_maps,
                const int *map_types, dock_grids **out);

/* Copies the node values of a grid set back to host memory in the layout of
 * load_grids (n_maps = n_type_maps + 2 for build_grids: type maps in the
 * order given, then electrostatic, then desolvation). */
int grids_read_maps(dock_ctx *ctx, const dock_grids *grids, float *maps_out);
int free_grids(dock_ctx *ctx, dock_grids *grids);

/* ---- ligand (Section II-A: atoms; rotatable bonds and rigid-body motion as
 * the degrees of freedom) ----
 * Host inputs: xyz [n_atoms][3] (A, the conformation at tau = 0), type codes,
 * partial charges, bonds [n_bonds][2] atom indices, rotatable[n_bonds] 0/1.
 * Builds on the host the rigid fragments, the torsion tree (root = largest
 * fragment), the pair list (atoms in different fragments, >= 4 bonds apart)
 * with per-pair coefficients, and uploads them.  Errors: n_atoms out of
 * 1..255, > 32 rotatable bonds, unknown type, bad bond index, disconnected
 * graph, rotatable bond in a ring, OOM. */
int load_ligand(dock_ctx *ctx, int n_atoms, const double *xyz, const int *type, const double *charge,
                int n_bonds, const int *bonds, const int *rotatable, dock_ligand **out);
/* Sizes of a loaded ligand (any pointer may be NULL). */
int ligand_info(const dock_ligand *lig, int *n_atoms, int *n_torsions, int *n_genes, int *n_pairs,
                int *n_fragments);
int free_ligand(dock_ctx *ctx, dock_ligand *lig);
/* Device bytes a loaded ligand holds (for admission by device memory). */
int ligand_device_bytes(const dock_ligand *lig, size_t *bytes);

/* ---- batched evaluation of genotypes (paper, Section II-A: population-parallel pose evaluation) ----
 * geno: device [B][G] FP32.  E: device [B] FP32 energies (kcal/mol).
 * grad: device [B][G] FP32, dE/dgenotype (the quaternion part is the
 * derivative through the normalisation, so it is orthogonal to q).
 * Every ligand atom type must have a map (DOCK_ERR_NOMAP).  B = 0 is a
 * no-op.  Deterministic: the same inputs give bit-identical outputs. */
int score_batch(dock_ctx *ctx, const dock_grids *grids, const dock_ligand *lig, const float *geno, int B,
                float *E, void *stream);
int score_grad_batch(dock_ctx *ctx, const dock_grids *grids, const dock_ligand *lig, const float *geno, int B,
                     float *E, float *grad, void *stream);
/* Atom coordinates of each genotype (Section IV-B: atom rotations along the
 * torsion tree), device [B][n_atoms][3] FP32 in input atom order. */
int pose_batch(dock_ctx *ctx, const dock_ligand *lig, const float *geno, int B, float *xyz, void *stream);

/* ---- the Lamarckian GA (Section II-A) ----
 * Runs params->nruns independent searches of params->pop_size individuals
 * until each has spent params->max_evals evaluations (checked at generation
 * boundaries).  Per generation: elitism, tournament selection, two-point
 * crossover, mutation, evaluation of the new individuals; the local search
 * (ADADELTA or Solis-Wets) on ls_count individuals drawn without
 * replacement, result written back; the per-run evaluation count grows by
 * (pop_size-1) + the local searches' evaluations (ls_count*ls_iters for
 * ADADELTA).  Random numbers: Philox4x32-10 keyed by seed, counter
 * (purpose<<16|draw, individual, generation, run).  Deterministic for a
 * given seed.  dock(): host outputs best_geno [nruns][G] (unit quaternion),
 * best_E [nruns] (FP64 re-score of best_geno), evals_used [nruns]; blocks
 * until done.  dock_async(): the same into device buffers (best_E32: the
 * FP32 energy the search kept), queued on `stream`; with Solis-Wets, whose
 * evaluation count is known only on the device, it also reads the runs'
 * counters back a few times (a stream synchronisation each) to decide how
 * many more generations to queue. */
int dock(dock_ctx *ctx, const dock_grids *grids, const dock_ligand *lig, const dock_params *params, uint64_t seed,
         float *best_geno, double *best_E, int64_t *evals_used);
int dock_async(dock_ctx *ctx, const dock_grids *grids, const dock_ligand *lig, const dock_params *params,
               uint64_t seed, float *best_geno, float *best_E32, double *best_E, int64_t *evals_used, void *stream);

/* ---- many ligands in one persistent launch ----
 * Docks n_ligs ligands against the same grids: every run of every ligand is
 * one task and one warp runs a whole task (all generations, children,
 * scores and local searches, the same operators and stream layout as
 * dock()), claiming tasks from a device counter, largest ligands first, so
 * ligands of uneven size share one launch.  seeds[k] (host, may be NULL =
 * k) keys ligand k's random stream.  Device outputs, row t = k * nruns + r:
 * best_geno [n_ligs*nruns][39] (genes 0..G_k-1 used, unit quaternion),
 * best_E32 [n_ligs*nruns] (may be NULL), best_E [n_ligs*nruns] (FP64
 * re-score), evals_used [n_ligs*nruns] (may be NULL).  Blocks until done.
 * A run's result depends only on its ligand, run index, seed and params, not
 * on the other ligands of the batch; it uses one-warp evaluation, so its
 * values may differ in the last bits from dock(), which spreads a local
 * search over several warps when runs are few. */
int dock_batch(dock_ctx *ctx, const dock_grids *grids, const dock_ligand *const *ligs, int n_ligs,
               const dock_params *params, const uint64_t *seeds, float *best_geno, float *best_E32, double *best_E,
               int64_t *evals_used, void *stream);

/* ---- autotuning: device time of candidate launch shapes ----
 * dock_tune times the kernel family `what` at each candidate launch shape
 * cand[0..n_cand-1] on the given inputs, `reps` launches each after one
 * untimed launch, and writes the mean device milliseconds per launch to
 * ms[i] (-1 where the candidate does not fit the device).  Nothing else is
 * kept: the caller picks a candidate and passes it in dock_params.
 *   DOCK_TUNE_LS_THREADS: the local search of dock() for ligs[0] (the
 *     paper's threads-per-block knob, Section V-B): params->nruns *
 *     ls_count chains (ls_method's search) of min(ls_iters, 50) iterations
 *     from an initial population; cand = threads per chain (32, 64, 128, 256).
 *   DOCK_TUNE_BATCH_WARPS: dock_batch over ligs[0..n_ligs-1] at params
 *     (give it a small max_evals); cand = warps per block (1, 2, 4).
 *   DOCK_TUNE_SCORE_BLOCKS: score_grad_batch of params->pop_size * nruns
 *     genotypes of ligs[0] (an initial population); cand = the register cap
 *     as DOCK_OPT_SCORE_BLOCKS values (1, 6, 8).  The context's own setting is
 *     restored afterwards.
 *   DOCK_TUNE_BATCH_BLOCKS: dock_batch as for DOCK_TUNE_BATCH_WARPS; cand =
 *     the register cap as DOCK_OPT_BATCH_BLOCKS values (3, 4).
 * Errors: unknown `what`, an invalid candidate value, n_cand < 1, reps < 1. */
#define DOCK_TUNE_LS_THREADS 1
#define DOCK_TUNE_BATCH_WARPS 2
#define DOCK_TUNE_SCORE_BLOCKS 3
#define DOCK_TUNE_BATCH_BLOCKS 4
int dock_tune(dock_ctx *ctx, const dock_grids *grids, const dock_ligand *const *ligs, int n_ligs,
              const dock_params *params, int what, const int *cand, int n_cand, int reps, double *ms);

/* Context options.  DOCK_OPT_SCORE_BLOCKS: register cap of the batched
 * scorers (score_batch, score_grad_batch) as the blocks of 128 threads per
 * SM the registers must leave room for: 1 (the compiler's choice, default),
 * 6 (<= 80 registers per thread) or 8 (<= 64).  It changes speed only, never
 * a result (the paper's register-use tuning, Section V-B).  Errors: unknown
 * option or value. */
#define DOCK_OPT_SCORE_BLOCKS 1
/* DOCK_OPT_BATCH_BLOCKS: register cap of dock_batch's and the server's
 * persistent docking kernel, as blocks of 128 threads per SM: 4 (<= 128
 * registers per thread, default) or 3 (<= 168; fewer spills, fewer warps).
 * A server takes the value set when server_create is called.  Speed only. */
#define DOCK_OPT_BATCH_BLOCKS 2
int dock_set_option(dock_ctx *ctx, int option, int value);
int dock_get_option(const dock_ctx *ctx, int option, int *value);

/* ---- device rates for the rooflines (no paper counterpart) ----
 * dock_microbench measures one rate of this device with a microbenchmark
 * kernel (best of three timed launches after a warm-up launch):
 *   DOCK_PEAK_FFMA: FP32 fused multiply-add throughput, TFLOP/s (2 FLOP each);
 *   DOCK_PEAK_EX2: special-function ex2.approx throughput, Gop/s;
 *   DOCK_PEAK_L2_READ: L2->SM load bandwidth over a 48 MB L2-resident
 *     buffer read with ld.global.cg, GB/s.
 * *value receives the rate.  Errors: unknown `what`, allocation failure. */
#define DOCK_PEAK_FFMA 1
#define DOCK_PEAK_EX2 2
#define DOCK_PEAK_L2_READ 3
int dock_microbench(dock_ctx *ctx, int what, double *value);

/* ---- serving: continuous batching of docking requests ----
 * A server keeps a persistent docking kernel fed from a queue: each request
 * (one ligand, its grids, params and seed) becomes nruns tasks; warps of the
 * running kernel pick tasks up as soon as they are submitted, so requests of
 * different sizes arriving while others run share the GPU at once.  The
 * queue lives in mapped host memory; idle warps poll it with a bounded wait.
 * After about a second with no task in progress the launch winds down as a
 * whole (every warp leaves and none claims again); server_submit and
 * server_poll relaunch the kernel when tasks are pending and none runs.  A
 * task's result depends only on its ligand, grids, params, seed and run
 * index (the same as dock_batch for them), not on what else is queued.
 * server_create: capacity = task slots (results of a task stay readable
 * until capacity more tasks have been submitted), max_atoms = largest
 * ligand accepted, pop_max = largest pop_size accepted.
 * server_submit: the ligand and grids must stay loaded until the request is
 * done; returns the request's first task number; DOCK_ERR_BUSY when the
 * slots it would reuse are still running.
 * server_poll: *done = 1 once all nruns tasks from first_task are finished.
 * server_result: host outputs best_geno [nruns][n_genes], best_E [nruns]
 * (FP64 re-score), evals_used [nruns] (each may be NULL).
 * server_cancel: withdraws the runs of a submitted request that no warp has
 * claimed yet (best effort: a run already running finishes normally); a
 * withdrawn run completes at once with evals_used 0 and best_E = +inf.
 * Errors: a task range not submitted.
 * server_destroy: asks the warps to leave, waits for them, frees. */
typedef struct dock_server dock_server;
int server_create(dock_ctx *ctx, int capacity, int max_atoms, int pop_max, dock_server **out);
int server_submit(dock_server *srv, const dock_grids *grids, const dock_ligand *lig, const dock_params *params,
                  uint64_t seed, int64_t *first_task);
int server_poll(dock_server *srv, int64_t first_task, int nruns, int *done);
int server_result(dock_server *srv, int64_t first_task, int nruns, int n_genes, float *best_geno, double *best_E,
                  int64_t *evals_used);
int server_cancel(dock_server *srv, int64_t first_task, int nruns);
int server_destroy(dock_server *srv);

/* ---- docking without device allocation ----
 * Not a step of the paper's method (it has no counterpart there): the same
 * docking as dock_async -- same kernels, same results for the same inputs --
 * for callers that must not allocate device memory during the call, such as
 * a host application that has handed all device memory to its own pool, a
 * plugin that is only ever given pointers, or a latency-critical loop in
 * which cudaMalloc/cudaFree (which can synchronise the device) are not
 * acceptable.  Its working buffers (two populations of nruns x pop_size
 * genotypes, their energies, the local-search picks and the per-run
 * counters; plus nruns floats when best_E32 is NULL) come from one fixed
 * array of DOCK_NOALLOC_SCRATCH_BYTES that every GPU loading the library
 * holds until the process exits.  It calls no cudaMalloc, cudaFree or
 * allocating library routine, and never the context's allocator.
 *  - A request needing more scratch than the array holds (about
 *    2 * nruns * pop_size * (4*G + 4) bytes) fails with DOCK_ERR_SIZE and a
 *    message giving the bytes needed.
 *  - dock_create looks up the array's device address (cudaGetSymbolAddress)
 *    with its device current.  That lookup loads the library's device code,
 *    which the CUDA runtime otherwise loads on first use, so the array is
 *    allocated when the context is created, not by a later call.  If that
 *    lookup failed, the first dock_async_noalloc call on the device repeats
 *    it; so create the context before any stream capture and before the
 *    application pools the rest of the device memory.  The context's device
 *    must be current when calling.
 *  - All calls share the one array and it keeps the last call's contents
 *    (the counters are cleared at the start of each call): calls that
 *    overlap on the GPU -- on different streams, or from different host
 *    threads -- race on it; serialise them.
 *  - It runs the ADADELTA local search only: ls_method != 0 fails with
 *    DOCK_ERR_INVALID.
 *  - It makes no host synchronisation either, and its launch sequence is
 *    fixed by the parameters, so a call can be captured into a CUDA graph
 *    (stream capture) and replayed; a replay recomputes the captured seed's
 *    docking into the same output pointers.  Capture after a first direct
 *    call with the same ligand, so that every kernel is loaded.
 * Outputs and arguments as dock_async. */
#define DOCK_NOALLOC_SCRATCH_BYTES (8u << 20)
int dock_async_noalloc(dock_ctx *ctx, const dock_grids *grids, const dock_ligand *lig, const dock_params *params,
                       uint64_t seed, float *best_geno, float *best_E32, double *best_E, int64_t *evals_used,
                       void *stream);

/* ---- operator-level entry points (the steps dock() composes) ---- all
 * pointers device, FP32 genes, runs r = 0..nruns-1 laid out [nruns][pop][G].
 * dock_init_population: generation-0 individuals (translation uniform in
 * the grid box, orientation uniform on the unit 3-sphere, torsions uniform
 * in [-pi, pi)); no evaluation.
 * dock_ga_children: next generation from pop_old/E_old (slot 0 = the best
 * old individual); no evaluation.  info (optional) [nruns][pop][5] int64:
 * parent 1, parent 2, crossover cut lo, cut hi, mutated-block mask.
 * dock_ls_picks: picks [nruns][n_ls], the individuals given a local search.
 * dock_local_search: ADADELTA from B start points x0 [B][G], iters
 * iterations each, `threads` per chain as in dock_params.ls_threads;
 * x_best [B][G] (unit quaternion) and E_best [B].
 * dock_local_search_trace: the same search, also recording every iteration
 * it of chain b: the point evaluated (x_trace [B][iters][G], quaternion as
 * stored, unnormalised), its gradient (g_trace [B][iters][G]) and energy
 * (E_trace [B][iters]).  The three trace pointers are given together or all
 * NULL (then it is dock_local_search).  Caller-owned device buffers.
 * dock_adadelta_step: one ADADELTA update (Zeiler 2012; the local search of
 * the memetic step, paper Section II-A) of B points [B][n_genes] in place,
 * given their gradients g [B][n_genes] and running averages Eg2, Edx2
 * [B][n_genes] (updated in place): per gene
 *     Eg2 <- rho Eg2 + (1 - rho) g^2
 *     dx  <- -sqrt(Edx2 + eps) / sqrt(Eg2 + eps) * g
 *     Edx2 <- rho Edx2 + (1 - rho) dx^2,   x <- x + dx,
 * then torsion genes (index >= 7) wrapped to [-pi, pi).  It is the update
 * dock_local_search applies after each evaluation, exposed on its own so it
 * can be checked gene by gene.  Errors: n_genes outside 7..39, rho outside
 * [0, 1), eps <= 0, B * n_genes > INT_MAX.
 * dock_philox: out[n][4] = Philox4x32-10(ctr[n][4], key = (key_lo, key_hi)). */
int dock_init_population(dock_ctx *ctx, const dock_grids *grids, int n_torsions, int pop, int nruns,
                         uint64_t seed, float *pop_out, void *stream);
int dock_ga_children(dock_ctx *ctx, int n_torsions, int pop, int nruns, const float *pop_old, const float *E_old,
                     uint64_t seed, uint32_t generation, const dock_params *params, float *pop_new,
                     int64_t *info, void *stream);
int dock_ls_picks(dock_ctx *ctx, int pop, int n_ls, int nruns, uint64_t seed, uint32_t generation, int *picks,
                  void *stream);
int dock_local_search(dock_ctx *ctx, const dock_grids *grids, const dock_ligand *lig, const float *x0, int B,
                      int iters, float rho, float eps, int threads, float *x_best, float *E_best, void *stream);
int dock_local_search_trace(dock_ctx *ctx, const dock_grids *grids, const dock_ligand *lig, const float *x0, int B,
                            int iters, float rho, float eps, int threads, float *x_best, float *E_best,
                            float *x_trace, float *g_trace, float *E_trace, void *stream);
int dock_adadelta_step(dock_ctx *ctx, int B, int n_genes, float rho, float eps, float *x, const float *g,
                       float *Eg2, float *Edx2, void *stream);
int dock_philox(dock_ctx *ctx, const uint32_t *ctr, int n, uint32_t key_lo, uint32_t key_hi, uint32_t *out,
                void *stream);
/* dock_solis_wets: the Solis-Wets local search (paper, Section II-A; Solis
 * and Wets 1981) from B start points x0 [B][G] (device), with their energies
 * E0 [B] (device; NULL = evaluate each start first, one more evaluation),
 * params->ls_iters iterations at most, the sw_* constants and ls_threads of
 * params.  Chain c draws its deviates from the Philox blocks
 * (6 << 16 | 10 it + j / 4, c, generation, run) under key = seed.  Outputs
 * (device): x_best [B][G] (quaternion normalised), E_best [B], evals [B]
 * (energies computed; may be NULL).  Errors: ls_iters > 6553. */
int dock_solis_wets(dock_ctx *ctx, const dock_grids *grids, const dock_ligand *lig, const float *x0,
                    const float *E0, int B, const dock_params *params, uint64_t seed, uint32_t run,
                    uint32_t generation, float *x_best, float *E_best, int64_t *evals, void *stream);

/* ---- tracing ----
 * With timing on, every kernel launch of dock/dock_async/score_* is
 * bracketed by CUDA events on its stream; dock_kernel_time() returns the
 * summed device time and launch count per kernel name ("dock_ls",
 * "dock_ga", "dock_init", "score", "score_grad", ...) since the last reset
 * (it synchronises the context's events).  dock_launch_count() counts every
 * kernel this context launched. */
int dock_set_timing(dock_ctx *ctx, int enable);
int dock_kernel_time(dock_ctx *ctx, const char *kernel, double *total_ms, int64_t *launches);
int dock_reset_timing(dock_ctx *ctx);
int64_t dock_launch_count(const dock_ctx *ctx);

#ifdef __cplusplus
}
#endif
#endif /* GB300_DOCK_H */
