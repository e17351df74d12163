// ga.cuh -- genetic operators, local-search sampling and the two local
// searches (ADADELTA; Solis-Wets, the paper's own) of the Lamarckian GA
// (paper, Section II-A), as warp-level device
// functions shared by the per-phase kernels (one docking, runs in parallel)
// and the persistent batch kernel (one warp runs a whole docking run).
//
// Genetic operators act on FP32 genes with one IEEE round-to-nearest
// operation per step (__fadd_rn & co., never contracted), so that given the
// same energies and the same Philox stream they are reproducible exactly by
// any IEEE single-precision implementation.
#pragma once

#include "eval.cuh"

namespace {

constexpr int kMaxLs = 256;
constexpr float kPiF = 3.14159265358979323846f;
constexpr float kTwoPiF = 6.28318530717958647692f;
enum : uint32_t { kInit = 1, kSelect = 2, kCross = 3, kMutate = 4, kLsPick = 5, kSw = 6 };

// Solis-Wets constants: step scale start / floor, expansion and contraction
// factors, the runs of successes / failures that trigger them, deviation
// half-widths per gene block at scale 1 (translation A, quaternion
// component, torsion rad).
struct SwConst {
    float rho0, rho_lo, expand, contract;
    int n_succ, n_fail;
    float step_t, step_q, step_tau;
};

struct GaConst {
    int pop, nruns, nt;
    float p_tour, p_cross, p_mut, trans_mut;
    uint2 key;
};

// Philox4x32-10 (Salmon et al., SC'11): ten rounds of two 32x32 -> 64-bit
// products with a Weyl-sequence key schedule.
__device__ __forceinline__ uint4 philox(uint4 c, uint2 k) {
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        if (r) {
            k.x += 0x9E3779B9u;
            k.y += 0xBB67AE85u;
        }
        const uint32_t hi0 = __umulhi(0xD2511F53u, c.x), lo0 = 0xD2511F53u * c.x;
        const uint32_t hi1 = __umulhi(0xCD9E8D57u, c.z), lo1 = 0xCD9E8D57u * c.z;
        c = make_uint4(hi1 ^ c.y ^ k.x, lo1, hi0 ^ c.w ^ k.y, lo0);
    }
    return c;
}

__device__ __forceinline__ uint4 draw4(uint2 key, uint32_t run, uint32_t gen, uint32_t entity, uint32_t purpose,
                                       uint32_t draw) {
    return philox(make_uint4((purpose << 16) | draw, entity, gen, run), key);
}

__device__ __forceinline__ uint32_t word(const uint4 &w, int i) {
    return i == 0 ? w.x : i == 1 ? w.y : i == 2 ? w.z : w.w;
}

// top 24 bits * 2^-24: exact in FP32
__device__ __forceinline__ float unif(uint32_t w) { return __fmul_rn((float)(w >> 8), 0x1p-24f); }
__device__ __forceinline__ uint32_t uidx(uint32_t w, uint32_t n) {
    return (uint32_t)(((unsigned long long)(w >> 8) * n) >> 24);
}

__device__ __forceinline__ float wrap_tau(float x) {
    if (x >= kPiF) x = __fsub_rn(x, kTwoPiF);
    else if (x < -kPiF) x = __fadd_rn(x, kTwoPiF);
    return x;
}

__device__ __forceinline__ int block_of_gene(int j) { return j < 3 ? j : (j < 7 ? 3 : j - 3); }

// Lexicographic (energy, index) minimum over the warp; every lane gets it.
__device__ __forceinline__ void warp_argmin(float &e, int &i) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const float e2 = __shfl_xor_sync(0xffffffffu, e, o);
        const int i2 = __shfl_xor_sync(0xffffffffu, i, o);
        if (e2 < e || (e2 == e && i2 < i)) {
            e = e2;
            i = i2;
        }
    }
}

__device__ int run_argmin(const float *E, int pop, int lane, float &best) {
    float be = INFINITY;
    int bi = 0x7fffffff;
    for (int i = lane; i < pop; i += 32) {
        const float e = E[i];
        if (e < be || (e == be && i < bi)) {
            be = e;
            bi = i;
        }
    }
    warp_argmin(be, bi);
    best = be;
    return bi;
}

// Generation-0 individual: translation uniform in the grid box, orientation
// uniform on S^3 (Marsaglia 1972: two points in the unit disc), torsions
// uniform in [-pi, pi).
__device__ void init_individual(const GaConst &C, const GridDev &G, uint32_t run, uint32_t slot, float *gene) {
    uint4 w = draw4(C.key, run, 0, slot, kInit, 0);
    gene[0] = __fadd_rn(G.box_lo[0], __fmul_rn(unif(w.x), G.box_len[0]));
    gene[1] = __fadd_rn(G.box_lo[1], __fmul_rn(unif(w.y), G.box_len[1]));
    gene[2] = __fadd_rn(G.box_lo[2], __fmul_rn(unif(w.z), G.box_len[2]));
    gene[3] = 1.f;
    gene[4] = gene[5] = gene[6] = 0.f;
    for (uint32_t att = 0; att < 32; ++att) {
        w = draw4(C.key, run, 0, slot, kInit, 1 + att);
        const float x1 = __fsub_rn(__fmul_rn(2.f, unif(w.x)), 1.f), x2 = __fsub_rn(__fmul_rn(2.f, unif(w.y)), 1.f);
        const float x3 = __fsub_rn(__fmul_rn(2.f, unif(w.z)), 1.f), x4 = __fsub_rn(__fmul_rn(2.f, unif(w.w)), 1.f);
        const float s1 = __fadd_rn(__fmul_rn(x1, x1), __fmul_rn(x2, x2));
        const float s2 = __fadd_rn(__fmul_rn(x3, x3), __fmul_rn(x4, x4));
        if (s1 < 1.f && s2 < 1.f && s2 > 0.f) {
            const float f = __fsqrt_rn(__fdiv_rn(__fsub_rn(1.f, s1), s2));
            gene[3] = x1;
            gene[4] = x2;
            gene[5] = __fmul_rn(x3, f);
            gene[6] = __fmul_rn(x4, f);
            break;
        }
    }
    for (int k = 0; k < C.nt; ++k) {
        if ((k & 3) == 0) w = draw4(C.key, run, 0, slot, kInit, 64 + (uint32_t)(k >> 2));
        gene[7 + k] = __fsub_rn(__fmul_rn(unif(word(w, k & 3)), kTwoPiF), kPiF);
    }
}

__device__ __forceinline__ int tournament(const float *E, int pop, float p_tour, uint4 w) {
    const int i1 = (int)uidx(w.x, (uint32_t)pop), i2 = (int)uidx(w.y, (uint32_t)pop);
    int better = i2, worse = i1;
    if (E[i1] < E[i2] || (E[i1] == E[i2] && i1 <= i2)) {
        better = i1;
        worse = i2;
    }
    return unif(w.z) < p_tour ? better : worse;
}


// Child s >= 1 of run r in generation gen, built by one warp into gs[]
// (shared memory): two tournaments, two-point crossover over gene blocks,
// per-block mutation.  dec[] (lane 0) gets parent 1, parent 2, cut lo, cut
// hi and the mutated-block mask.
__device__ void make_child(const GaConst &C, uint32_t gen, int r, int s, const float *__restrict__ old,
                           const float *__restrict__ Eo, float *gs, int lane, long long *dec) {
    const int Gn = 7 + C.nt, nblk = 4 + C.nt;
    int p1 = 0, p2 = 0, lo = 0, hi = 0;
    unsigned long long mask = 0;
    if (lane == 0) {
        p1 = tournament(Eo, C.pop, C.p_tour, draw4(C.key, r, gen, s, kSelect, 0));
        p2 = tournament(Eo, C.pop, C.p_tour, draw4(C.key, r, gen, s, kSelect, 1));
        const uint4 w = draw4(C.key, r, gen, s, kCross, 0);
        if (unif(w.x) < C.p_cross) {
            const int c1 = (int)uidx(w.y, (uint32_t)nblk), c2 = (int)uidx(w.z, (uint32_t)nblk);
            lo = min(c1, c2);
            hi = max(c1, c2);
        }
        uint4 m = make_uint4(0, 0, 0, 0);
        for (int b = 0; b < nblk; ++b) {
            if ((b & 3) == 0) m = draw4(C.key, r, gen, s, kMutate, (uint32_t)(b >> 2));
            if (unif(word(m, b & 3)) < C.p_mut) mask |= 1ull << b;
        }
    }
    p1 = __shfl_sync(0xffffffffu, p1, 0);
    p2 = __shfl_sync(0xffffffffu, p2, 0);
    lo = __shfl_sync(0xffffffffu, lo, 0);
    hi = __shfl_sync(0xffffffffu, hi, 0);
    mask = __shfl_sync(0xffffffffu, mask, 0);
    for (int j = lane; j < Gn; j += 32) {
        const int b = block_of_gene(j);
        gs[j] = old[(size_t)((b >= lo && b < hi) ? p2 : p1) * Gn + j];
    }
    __syncwarp();
    for (int b = lane; b < nblk; b += 32) {
        if (!((mask >> b) & 1ull)) continue;
        const uint4 v = draw4(C.key, r, gen, s, kMutate, 16 + (uint32_t)b);
        if (b < 3) {
            const float delta = __fsub_rn(__fmul_rn(unif(v.x), __fmul_rn(2.f, C.trans_mut)), C.trans_mut);
            gs[b] = __fadd_rn(gs[b], delta);
        } else if (b == 3) {
            // q <- normalise((1, v) (x) q), v uniform in [-1, 1)^3
            const float vx = __fsub_rn(__fmul_rn(2.f, unif(v.x)), 1.f);
            const float vy = __fsub_rn(__fmul_rn(2.f, unif(v.y)), 1.f);
            const float vz = __fsub_rn(__fmul_rn(2.f, unif(v.z)), 1.f);
            const float qw = gs[3], qx = gs[4], qy = gs[5], qz = gs[6];
            const float nw = __fsub_rn(__fsub_rn(__fsub_rn(qw, __fmul_rn(vx, qx)), __fmul_rn(vy, qy)), __fmul_rn(vz, qz));
            const float nx = __fsub_rn(__fadd_rn(__fadd_rn(qx, __fmul_rn(vx, qw)), __fmul_rn(vy, qz)), __fmul_rn(vz, qy));
            const float ny = __fadd_rn(__fadd_rn(__fsub_rn(qy, __fmul_rn(vx, qz)), __fmul_rn(vy, qw)), __fmul_rn(vz, qx));
            const float nz = __fadd_rn(__fsub_rn(__fadd_rn(qz, __fmul_rn(vx, qy)), __fmul_rn(vy, qx)), __fmul_rn(vz, qw));
            const float n = __fsqrt_rn(__fadd_rn(__fadd_rn(__fadd_rn(__fmul_rn(nw, nw), __fmul_rn(nx, nx)), __fmul_rn(ny, ny)),
                                                 __fmul_rn(nz, nz)));
            gs[3] = __fdiv_rn(nw, n);
            gs[4] = __fdiv_rn(nx, n);
            gs[5] = __fdiv_rn(ny, n);
            gs[6] = __fdiv_rn(nz, n);
        } else {
            const float delta = __fsub_rn(__fmul_rn(unif(v.x), kTwoPiF), kPiF);
            gs[b + 3] = wrap_tau(__fadd_rn(gs[b + 3], delta));
        }
    }
    __syncwarp();
    dec[0] = p1; dec[1] = p2; dec[2] = lo; dec[3] = hi; dec[4] = (long long)mask;
}

// The local-search sample of run r in generation gen: the first n_ls entries
// of a partial Fisher-Yates shuffle of 0..pop-1, kept as a list of displaced
// positions instead of a pop-sized array.  One thread.
__device__ void ls_picks_one(int pop, int n_ls, uint2 key, uint32_t r, uint32_t gen, int *picks) {
    int pos[2 * kMaxLs], val[2 * kMaxLs], cnt = 0;
    for (int k = 0; k < n_ls; ++k) {
        const uint32_t w = draw4(key, r, gen, k, kLsPick, 0).x;
        const int j = k + (int)uidx(w, (uint32_t)(pop - k));
        int vk = k, vj = j, ik = -1, ij = -1;
        for (int e = 0; e < cnt; ++e) {
            if (pos[e] == k) { vk = val[e]; ik = e; }
            if (pos[e] == j) { vj = val[e]; ij = e; }
        }
        if (ik < 0) { ik = cnt++; pos[ik] = k; }
        val[ik] = vj;
        if (j != k) {
            if (ij < 0) { ij = cnt++; pos[ij] = j; }
            val[ij] = vk;
        }
        picks[k] = vj;
    }
}

__device__ __forceinline__ void adadelta(float &x, float g, float &eg2, float &edx2, float rho, float eps) {
    eg2 = fmaf(rho, eg2, (1.f - rho) * g * g);
    const float dx = -sqrtf(edx2 + eps) * rsqrtf(eg2 + eps) * g;
    edx2 = fmaf(rho, edx2, (1.f - rho) * dx * dx);
    x += dx;
}

__device__ __forceinline__ float wrap_any(float x) {
    return x - kTwoPiF * floorf((x + kPiF) * (1.f / kTwoPiF));
}

// Optional per-iteration record of one ADADELTA chain: the point evaluated
// at iteration it (x[it][G]), its gradient (g[it][G]) and energy (E[it]).
// Null pointers record nothing.
struct LsTrace {
    float *x, *g, *E;
};

// ADADELTA from xi for iters iterations by a team of W warps (warp 0 owns
// the genes: lane l holds genes l and l + 32); the best point seen, its
// quaternion normalised, is written to xo (which may alias xi).  Returns the
// best energy (on warp 0).  tr (optional) records every iteration.
template <int W>
__device__ float ls_chain(const LigandDev &L, const GridDev &G, float *ws, const EvalLayout &Y,
                          const dev::Team<W> &tm, const float *xi, float *xo, int iters, float rho, float eps,
                          LsTrace tr = LsTrace{nullptr, nullptr, nullptr}) {
    const int Gn = L.n_genes;
    // warp 0 owns the genes: lane l holds genes l and l + 32
    const bool w0 = tm.warp() == 0;
    const int lane = threadIdx.x & 31, j0 = lane, j1 = lane + 32;
    float x0 = 0.f, x1 = 0.f;
    if (w0) {
        x0 = j0 < Gn ? xi[j0] : 0.f;
        x1 = j1 < Gn ? xi[j1] : 0.f;
    }
    float b0 = x0, b1 = x1, best = INFINITY;
    float g2a = 0.f, g2b = 0.f, d2a = 0.f, d2b = 0.f;
    for (int it = 0; it < iters; ++it) {
        if (w0) {
            if (j0 < Gn) ws[Y.geno + j0] = x0;
            if (j1 < Gn) ws[Y.geno + j1] = x1;
        }
        // the evaluator's warp 0 reads the genes after a __syncwarp; the
        // other warps read them only after the team's barriers
        const float e = dev::eval_team<W, true>(L, G, ws, Y, tm);
        if (w0 && tr.x) {
            float *tx = tr.x + (size_t)it * Gn, *tg = tr.g + (size_t)it * Gn;
            if (j0 < Gn) { tx[j0] = x0; tg[j0] = ws[Y.grad + j0]; }
            if (j1 < Gn) { tx[j1] = x1; tg[j1] = ws[Y.grad + j1]; }
            if (lane == 0) tr.E[it] = e;
        }
        if (w0) {
            if (e < best) {
                best = e;
                b0 = x0;
                b1 = x1;
            }
            if (j0 < Gn) {
                adadelta(x0, ws[Y.grad + j0], g2a, d2a, rho, eps);
                if (j0 >= 7) x0 = wrap_any(x0);
            }
            if (j1 < Gn) {
                adadelta(x1, ws[Y.grad + j1], g2b, d2b, rho, eps);
                x1 = wrap_any(x1);
            }
        }
    }
    // best point, quaternion normalised (FP32, fixed order)
    if (w0) {
        const float q3 = __shfl_sync(0xffffffffu, b0, 3), q4 = __shfl_sync(0xffffffffu, b0, 4);
        const float q5 = __shfl_sync(0xffffffffu, b0, 5), q6 = __shfl_sync(0xffffffffu, b0, 6);
        const float n = sqrtf(((q3 * q3 + q4 * q4) + q5 * q5) + q6 * q6);
        if (j0 >= 3 && j0 < 7 && n > 0.f) b0 = b0 / n;
        if (j0 < Gn) xo[j0] = b0;
        if (j1 < Gn) xo[j1] = b1;
    }
    return best;
}


// Torsion wrap to [-pi, pi) for any finite x, single rounded operations.
__device__ __forceinline__ float wrap_any_rn(float x) {
    const float k = floorf(__fdiv_rn(__fadd_rn(x, kPiF), kTwoPiF));
    return __fsub_rn(x, __fmul_rn(kTwoPiF, k));
}

// Solis-Wets (Solis and Wets 1981: adaptive random search with a bias term)
// from xi with energy e0 (NaN: evaluated first) by a team of W warps; warp 0
// owns the genes (lane l: genes l and l + 32).  Each iteration draws
//     d_j = b_j + rho * step(block of j) * u_j,   u_j uniform in [-1, 1)
// (u_j: word j mod 4 of the Philox block (kSw << 16 | 10 it + j / 4, entity,
// gen, run)), tries x + d, then x - d if that was not lower.  A success moves
// x (b <- 0.2 b + 0.4 d forward, b <- b - 0.4 d backward), a failure halves
// b; n_succ successes in a row scale rho by expand, n_fail failures by
// contract.  Stops after iters iterations or once rho < rho_lo.  Gene
// arithmetic is single rounded FP32 operations in a fixed order, so given
// the same accept decisions any IEEE implementation reproduces the points.
// Writes x (quaternion normalised) to xo, which may alias xi; returns its
// energy; evals = energies computed.  Every thread of the team returns the
// same values.
template <int W>
__device__ float sw_chain(const LigandDev &L, const GridDev &G, float *ws, const EvalLayout &Y, const dev::Team<W> &tm,
                          const float *xi, float e0, float *xo, int iters, const SwConst &S, uint2 key, uint32_t run,
                          uint32_t gen, uint32_t entity, long long &evals) {
    const int Gn = L.n_genes;
    const bool w0 = tm.warp() == 0;
    const int lane = threadIdx.x & 31, j0 = lane, j1 = lane + 32;
    const bool h0 = j0 < Gn, h1 = j1 < Gn;
    float x0 = 0.f, x1 = 0.f, b0 = 0.f, b1 = 0.f, d0 = 0.f, d1 = 0.f, y0 = 0.f, y1 = 0.f;
    if (w0) {
        x0 = h0 ? xi[j0] : 0.f;
        x1 = h1 ? xi[j1] : 0.f;
    }
    const float s0 = j0 < 3 ? S.step_t : (j0 < 7 ? S.step_q : S.step_tau), s1 = S.step_tau;
    float *gs = ws + Y.geno;
    long long n = 0;
    float E = e0;
    if (isnan(e0)) {
        if (w0) {
            if (h0) gs[j0] = x0;
            if (h1) gs[j1] = x1;
        }
        E = dev::eval_team<W, false>(L, G, ws, Y, tm);
        ++n;
    }
    float rho = S.rho0;
    int ns = 0, nf = 0, it = 0;
    for (; it < iters && rho >= S.rho_lo; ++it) {
        if (w0) {
            const float sr0 = __fmul_rn(rho, s0), sr1 = __fmul_rn(rho, s1);
            const uint4 wa = draw4(key, run, gen, entity, kSw, (uint32_t)(10 * it + (j0 >> 2)));
            d0 = __fadd_rn(b0, __fmul_rn(sr0, __fsub_rn(__fmul_rn(2.f, unif(word(wa, j0 & 3))), 1.f)));
            if (h1) {
                const uint4 wb = draw4(key, run, gen, entity, kSw, (uint32_t)(10 * it + (j1 >> 2)));
                d1 = __fadd_rn(b1, __fmul_rn(sr1, __fsub_rn(__fmul_rn(2.f, unif(word(wb, j1 & 3))), 1.f)));
            }
            y0 = __fadd_rn(x0, d0);
            y1 = __fadd_rn(x1, d1);
            if (j0 >= 7) y0 = wrap_any_rn(y0);
            y1 = wrap_any_rn(y1);
            if (h0) gs[j0] = y0;
            if (h1) gs[j1] = y1;
        }
        const float ef = dev::eval_team<W, false>(L, G, ws, Y, tm);
        ++n;
        bool ok = ef < E;
        if (ok) {
            E = ef;
            if (w0) {
                x0 = y0;
                x1 = y1;
                b0 = __fadd_rn(__fmul_rn(0.2f, b0), __fmul_rn(0.4f, d0));
                b1 = __fadd_rn(__fmul_rn(0.2f, b1), __fmul_rn(0.4f, d1));
            }
        } else {
            if (w0) {
                y0 = __fsub_rn(x0, d0);
                y1 = __fsub_rn(x1, d1);
                if (j0 >= 7) y0 = wrap_any_rn(y0);
                y1 = wrap_any_rn(y1);
                if (h0) gs[j0] = y0;
                if (h1) gs[j1] = y1;
            }
            const float eb = dev::eval_team<W, false>(L, G, ws, Y, tm);
            ++n;
            ok = eb < E;
            if (ok) {
                E = eb;
                if (w0) {
                    x0 = y0;
                    x1 = y1;
                    b0 = __fsub_rn(b0, __fmul_rn(0.4f, d0));
                    b1 = __fsub_rn(b1, __fmul_rn(0.4f, d1));
                }
            } else if (w0) {
                b0 = __fmul_rn(0.5f, b0);
                b1 = __fmul_rn(0.5f, b1);
            }
        }
        if (ok) {
            ++ns;
            nf = 0;
        } else {
            ++nf;
            ns = 0;
        }
        if (ns >= S.n_succ) {
            rho = __fmul_rn(rho, S.expand);
            ns = 0;
        } else if (nf >= S.n_fail) {
            rho = __fmul_rn(rho, S.contract);
            nf = 0;
        }
    }
    if (w0) {
        const float q3 = __shfl_sync(0xffffffffu, x0, 3), q4 = __shfl_sync(0xffffffffu, x0, 4);
        const float q5 = __shfl_sync(0xffffffffu, x0, 5), q6 = __shfl_sync(0xffffffffu, x0, 6);
        const float qn = __fsqrt_rn(__fadd_rn(__fadd_rn(__fadd_rn(__fmul_rn(q3, q3), __fmul_rn(q4, q4)), __fmul_rn(q5, q5)),
                                              __fmul_rn(q6, q6)));
        if (j0 >= 3 && j0 < 7 && qn > 0.f) x0 = __fdiv_rn(x0, qn);
        if (h0) xo[j0] = x0;
        if (h1) xo[j1] = x1;
    }
    evals = n;
    return E;
}

}  // namespace
