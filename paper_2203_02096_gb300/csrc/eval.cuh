// eval.cuh -- a team of W warps evaluates the energy (and gradient) of one
// genotype.
//
// Steps (paper, Section II-A / IV-B): genotype -> pose by rotations along
// the torsion tree; particle-grid energy by trilinear reads of the receptor
// maps; intramolecular pair energy (vdW / H-bond, screened Coulomb,
// desolvation); then the analytic genotype gradient.
//
// W = 1 (one warp per genotype) serves the throughput paths, where there are
// many more genotypes than warps; W = 2..8 serves the local search when the
// independent chains are too few to fill the GPU: the team splits atoms,
// pairs and force gathers, like the paper's threads-per-block knob.
//
// GB300 layout: pose, forces, torques and staged map cells live in shared
// memory; ligand constants and pair records come through L1 (read-only
// path); each atom-map read is one 32-byte cell (two adjacent quads) of the
// z-column quad grid copy, L2-resident.
// Every reduction has a fixed order (strided partial sums, xor butterflies,
// then warps in index order), so results are bit-reproducible run to run.
#pragma once

#include "internal.h"

namespace dev {

constexpr float kDielA = -8.5525f;
constexpr float kDielB = (float)(78.4 + 8.5525);
constexpr float kDielK = 7.7839f;
// exponents in base 2: e^{-a x} = 2^{-a log2(e) x}
constexpr double kLog2e = 1.4426950408889634;
constexpr float kDielLB2 = (float)(0.003627 * (78.4 + 8.5525) * kLog2e);
constexpr float kDielDeps = (float)((78.4 + 8.5525) * 7.7839 * 0.003627 * (78.4 + 8.5525));
constexpr float kHalfInvSig2L2 = (float)(kLog2e / (2.0 * 3.6 * 3.6));
constexpr float kInvSig2 = (float)(1.0 / (3.6 * 3.6));
constexpr float kCut2 = 64.0f;
constexpr float kFloor2 = 0.25f;
constexpr float kKout = 10.0f;

template <typename T>
__device__ __forceinline__ T ldg(const T *p) { return __ldg(p); }

// 2^x and 1/x by the special-function unit (ex2.approx / rcp.approx, about
// 2 ulp; inputs far below 0 give 0).
__device__ __forceinline__ float ex2_approx(float x) {
    float y;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}
__device__ __forceinline__ float rcp_approx(float x) {
    float y;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

// Paired FP32 arithmetic (sm_100-family add/mul/fma .f32x2 through the
// __fadd2_rn / __fmul2_rn / __ffma2_rn intrinsics): one issue slot for two
// operations, each rounded like its scalar _rn form.  A paired product that
// feeds a paired add can still be fused by the code generator in some
// kernels and not in others, so results would depend on the kernel: the
// evaluator never adds a paired product with add2 -- products enter sums only
// through explicit fma2/fmaf or after scalar rounding (__fadd_rn).
typedef float2 f32x2;
__device__ __forceinline__ f32x2 pk2(float a, float b) { return make_float2(a, b); }
__device__ __forceinline__ f32x2 dup2(float a) { return make_float2(a, a); }
__device__ __forceinline__ f32x2 add2(f32x2 a, f32x2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ f32x2 mul2(f32x2 a, f32x2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ f32x2 fma2(f32x2 a, f32x2 b, f32x2 c) { return __ffma2_rn(a, b, c); }
// a - b as fma(b, -1, a): the same single rounding
__device__ __forceinline__ f32x2 sub2(f32x2 a, f32x2 b) { return __ffma2_rn(b, make_float2(-1.f, -1.f), a); }

// W warps evaluating one genotype.  W = 1: a warp, possibly one of several
// independent teams in a block; W > 1: the whole block is the team.
template <int W>
struct Team {
    static constexpr int kSize = 32 * W;
    int rank;  // 0 .. 32W-1
    __device__ __forceinline__ explicit Team(int r) : rank(r) {}
    __device__ __forceinline__ int lane() const { return rank & 31; }
    __device__ __forceinline__ int warp() const { return rank >> 5; }
    __device__ __forceinline__ void sync() const {
        if (W == 1) __syncwarp();
        else __syncthreads();
    }
};

// Where an atom sits in the grid: cell index, in-cell fractions, clamping
// and the out-of-box penalty (energy and its gradient in kcal/mol/A).
struct CellPos {
    long long cell;  // quad index of the cell's lower z plane within a map
    float fx, fy, fz;
    bool cx, cy, cz;
    float pen, gpx, gpy, gpz;
};

__device__ __forceinline__ void clamp_axis(float u, int n, float h, int &i, float &f, bool &cl, float &pen, float &gp) {
    float d = 0.f;
    cl = false;
    const float top = (float)(n - 1);
    if (u < 0.f) { d = u; u = 0.f; cl = true; }
    else if (u > top) { d = u - top; u = top; cl = true; }
    int k = (int)floorf(u);
    k = k > n - 2 ? n - 2 : k;
    i = k;
    f = u - (float)k;
    const float dh = d * h;
    pen += kKout * dh * dh;
    gp = 2.f * kKout * dh;
}

__device__ __forceinline__ void locate(const GridDev &G, float ux, float uy, float uz, CellPos &c) {
    int ix, iy, iz;
    c.pen = 0.f;
    clamp_axis(ux, G.nx, G.h, ix, c.fx, c.cx, c.pen, c.gpx);
    clamp_axis(uy, G.ny, G.h, iy, c.fy, c.cy, c.pen, c.gpy);
    clamp_axis(uz, G.nz, G.h, iz, c.fz, c.cz, c.pen, c.gpz);
    c.cell = ((long long)iy * (G.nx - 1) + ix) * G.nz + iz;
}

// The 8 corner values of map m in the located cell: quads iz and iz + 1.
struct Cell8 {
    float4 a, b;
};

// Trilinear read in the located cell; derivatives are with respect to the
// in-cell fractions.
template <bool GRAD>
__device__ __forceinline__ float trilinear(const Cell8 &v, const CellPos &c, float &gx, float &gy, float &gz) {
    const float4 a = v.a, b = v.b;
    const float ax = a.y - a.x, az = a.w - a.z, bx = b.y - b.x, bz = b.w - b.z;
    const float x00 = fmaf(c.fx, ax, a.x), x10 = fmaf(c.fx, az, a.z);
    const float x01 = fmaf(c.fx, bx, b.x), x11 = fmaf(c.fx, bz, b.z);
    const float y0 = fmaf(c.fy, x10 - x00, x00), y1 = fmaf(c.fy, x11 - x01, x01);
    if (GRAD) {
        const float d0 = fmaf(c.fy, az - ax, ax), d1 = fmaf(c.fy, bz - bx, bx);
        gx = fmaf(c.fz, d1 - d0, d0);
        const float e0 = x10 - x00, e1 = x11 - x01;
        gy = fmaf(c.fz, e1 - e0, e0);
        gz = y1 - y0;
    }
    return fmaf(c.fz, y1 - y0, y0);
}

// An atom's grid cells and where it sits in them.
struct AtomCells {
    CellPos c;
    Cell8 t, e, d;
    float q;
};


// Asynchronous staging of an atom's three map cells (type, electrostatic,
// desolvation; two float4 each) into shared memory with cp.async: 16-byte
// global->shared copies that use no registers, so every atom's L2 reads are
// in flight while the pair rounds run.  The copying thread waits for its own
// copies (cp.async.wait_all) before it reads them back.
__device__ __forceinline__ void cp_async16(void *smem, const void *gmem) {
    const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(s), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;" ::: "memory"); }

__device__ __forceinline__ void atom_stage(const GridDev &G, int map_t, float ux, float uy, float uz, float4 *dst) {
    CellPos c;
    locate(G, ux, uy, uz, c);
    const float4 *bt = G.cells + (size_t)map_t * G.mstride + c.cell;
    const float4 *be = G.cells + (size_t)G.emap * G.mstride + c.cell;
    const float4 *bd = G.cells + (size_t)G.dmap * G.mstride + c.cell;
    cp_async16(dst + 0, bt);
    cp_async16(dst + 1, bt + 1);
    cp_async16(dst + 2, be);
    cp_async16(dst + 3, be + 1);
    cp_async16(dst + 4, bd);
    cp_async16(dst + 5, bd + 1);
}

// The staged cells of an atom back as AtomCells (its cell position located
// again from the same coordinates).
__device__ __forceinline__ void atom_unstage(const GridDev &G, float q, float ux, float uy, float uz,
                                             const float4 *src, AtomCells &A) {
    locate(G, ux, uy, uz, A.c);
    A.t = Cell8{src[0], src[1]};
    A.e = Cell8{src[2], src[3]};
    A.d = Cell8{src[4], src[5]};
    A.q = q;
}

// Energy of one atom (type map + q * electrostatic + |q| * desolvation +
// out-of-box penalty) and dE/dx, from its fetched cells.
template <bool GRAD>
__device__ __forceinline__ float atom_grid_energy(const GridDev &G, const AtomCells &A, float3 &g) {
    float tx, ty, tz, ex, ey, ez, dx, dy, dz;
    const float q = A.q, aq = fabsf(q);
    const float vt = trilinear<GRAD>(A.t, A.c, tx, ty, tz);
    const float ve = trilinear<GRAD>(A.e, A.c, ex, ey, ez);
    const float vd = trilinear<GRAD>(A.d, A.c, dx, dy, dz);
    if (GRAD) {
        const float sx = A.c.cx ? 0.f : G.inv_h, sy = A.c.cy ? 0.f : G.inv_h, sz = A.c.cz ? 0.f : G.inv_h;
        g.x = fmaf(sx, fmaf(aq, dx, fmaf(q, ex, tx)), A.c.gpx);
        g.y = fmaf(sy, fmaf(aq, dy, fmaf(q, ey, ty)), A.c.gpy);
        g.z = fmaf(sz, fmaf(aq, dz, fmaf(q, ez, tz)), A.c.gpz);
    }
    return fmaf(aq, vd, fmaf(q, ve, vt)) + A.c.pen;
}

// Intramolecular pair energies of two pairs at once (a lane's rounds d and
// d + 1).  Per pair, with coefficients (c12, cn, qq, ds): vdW pairs carry
// cn = c6 >= 0 (E = c12/r^12 - c6/r^6), H-bond pairs cn = -c10 < 0 (E =
// c12/r^12 - c10/r^10); qq = w_el 332.06 q_i q_j; ds = w_ds (S_i V_j + S_j
// V_i).  r2a, r2b: squared distances; C, N, Q, D: the two pairs' c12, cn, qq,
// ds.  Returns both energies; with GRAD, sa, sb = (dE/dr)/r (0 below the
// floor).
template <bool GRAD>
__device__ __forceinline__ f32x2 pair_energy2(float r2a, float r2b, f32x2 C, f32x2 N, f32x2 Q, f32x2 D, float &sa,
                                              float &sb) {
    const float r2ea = fmaxf(r2a, kFloor2), r2eb = fmaxf(r2b, kFloor2);
    const f32x2 R2E = pk2(r2ea, r2eb), RI = pk2(rsqrtf(r2ea), rsqrtf(r2eb));
    const f32x2 R = mul2(R2E, RI);
    const f32x2 RI2 = mul2(RI, RI), RI4 = mul2(RI2, RI2), RI6 = mul2(RI4, RI2), RI12 = mul2(RI6, RI6);
    const f32x2 RI10 = mul2(RI6, RI4);
    const float na = N.x, nb = N.y, r6a = RI6.x, r6b = RI6.y, r10a = RI10.x, r10b = RI10.y;
    const bool hba = na < 0.f, hbb = nb < 0.f;
    const f32x2 RK = pk2(hba ? r10a : r6a, hbb ? r10b : r6b);  // r^-10 or r^-6
    const f32x2 NCN = pk2(-fabsf(na), -fabsf(nb));
    const f32x2 EV = fma2(C, RI12, mul2(NCN, RK));
    // sigmoidal dielectric eps = A + B / den, den = 1 + k exp(-lambda B r):
    // eps = D / den with D = A den + B, so one reciprocal rr = 1 / (den D)
    // gives 1/eps = den^2 rr and eps'/eps = B k lambda B e rr
    const f32x2 T = mul2(R, dup2(-kDielLB2));
    const f32x2 EX = pk2(ex2_approx(T.x), ex2_approx(T.y));
    const f32x2 DEN = fma2(dup2(kDielK), EX, dup2(1.f));
    const f32x2 DD = mul2(DEN, fma2(dup2(kDielA), DEN, dup2(kDielB)));
    const f32x2 RR = pk2(rcp_approx(DD.x), rcp_approx(DD.y));
    const f32x2 INV_EPS = mul2(mul2(DEN, DEN), RR);
    // every product rounded on its own (paired instructions are never
    // contracted), so an energy has the same bits with and without the
    // gradient
    const f32x2 EEL = mul2(mul2(Q, RI), INV_EPS);
    const f32x2 U = mul2(R2E, dup2(-kHalfInvSig2L2));
    const f32x2 EDS = mul2(D, pk2(ex2_approx(U.x), ex2_approx(U.y)));
    if (GRAD) {
        // dE/dr = dv - eel (1/r + eps'/eps) - eds r / sigma^2, the last two
        // terms fused into the sum
        const f32x2 KN = pk2(hba ? -10.f : -6.f, hbb ? -10.f : -6.f);
        const f32x2 DV = mul2(fma2(mul2(C, dup2(-12.f)), RI12, mul2(mul2(KN, NCN), RK)), RI);
        const f32x2 Y = fma2(mul2(dup2(kDielDeps), EX), RR, RI);  // 1/r + eps'/eps
        const f32x2 T = fma2(mul2(EDS, R), dup2(-kInvSig2), fma2(mul2(EEL, dup2(-1.f)), Y, DV));
        const f32x2 SS = mul2(T, RI);
        sa = r2a >= kFloor2 ? SS.x : 0.f;
        sb = r2b >= kFloor2 ? SS.y : 0.f;
    }
    return pk2(__fadd_rn(__fadd_rn(EV.x, EEL.x), EDS.x), __fadd_rn(__fadd_rn(EV.y, EEL.y), EDS.y));
}

__device__ __forceinline__ float warp_sum(float v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// Sums over groups of 2^kl consecutive lanes, several values per level so
// their shuffles overlap.
__device__ __forceinline__ void group_sum3(float &a, float &b, float &c, int kl) {
    for (int o = (1 << kl) >> 1; o > 0; o >>= 1) {
        a += __shfl_xor_sync(0xffffffffu, a, o);
        b += __shfl_xor_sync(0xffffffffu, b, o);
        c += __shfl_xor_sync(0xffffffffu, c, o);
    }
}

__device__ __forceinline__ void group_sum6(float &a, float &b, float &c, float &d, float &e, float &f, int kl) {
    for (int o = (1 << kl) >> 1; o > 0; o >>= 1) {
        a += __shfl_xor_sync(0xffffffffu, a, o);
        b += __shfl_xor_sync(0xffffffffu, b, o);
        c += __shfl_xor_sync(0xffffffffu, c, o);
        d += __shfl_xor_sync(0xffffffffu, d, o);
        e += __shfl_xor_sync(0xffffffffu, e, o);
        f += __shfl_xor_sync(0xffffffffu, f, o);
    }
}

// Team-wide sum, same bits on every thread: warp butterflies, then the warps'
// partials added in warp order.  Its barrier also publishes every earlier
// shared-memory write of the team; `red` is not rewritten before two more
// team barriers have passed.
template <int W>
__device__ __forceinline__ float team_sum(const Team<W> &tm, float v, float *red) {
    v = warp_sum(v);
    if (W == 1) {
        __syncwarp();
        return v;
    }
    if (tm.lane() == 0) red[tm.warp()] = v;
    tm.sync();
    float s = red[0];
#pragma unroll
    for (int w = 1; w < W; ++w) s += red[w];
    return s;
}

// log2 of the largest power of two k <= kmax with items * k <= team size.
__device__ __forceinline__ int lanes_log2(int items, int team, int kmax) {
    int kl = 0;
    while ((2 << kl) <= kmax && items * (2 << kl) <= team) ++kl;
    return kl;
}

// Evaluates the genotype stored at ws[Y.geno ...], which only warp 0 needs
// to have written (and, for W > 1, only warp 0 may have written since the
// team's previous barrier).  Returns E on every thread of the team; with
// GRAD, dE/dgenotype is left at ws[Y.grad ...].
template <int W, bool GRAD>
__device__ float eval_team(const LigandDev &L, const GridDev &G, float *ws, const EvalLayout &Y, const Team<W> &tm) {
    constexpr int S = Team<W>::kSize;
    const int r = tm.rank, lane = tm.lane();
    const float *geno = ws + Y.geno;
    float4 *M = reinterpret_cast<float4 *>(ws + Y.M);
    // atom positions, pair-major: XP[j] = (x_j, x_j', y_j, y_j'), ZP[j] =
    // (z_j, z_j'), j' = the next atom of j's block (cyclic), so that a lane's
    // partners of rounds d and d + 1 come in one read as ready pairs
    float4 *XP = reinterpret_cast<float4 *>(ws + Y.x);
    float2 *ZP = reinterpret_cast<float2 *>(ws + Y.z);
    auto pos = [&](int i) {
        const float4 v = XP[i];
        return make_float3(v.x, v.z, ZP[i].x);
    };
    float4 *PF = reinterpret_cast<float4 *>(ws + Y.pf);
    float *red = ws + Y.red;
    const int T = L.n_tors, N = L.n_atoms, NB = L.nb8;
    // partial-force rows of the W > 1 groups: NB + 4 float4 apart, so the two
    // rows a quarter-warp reads at once fall on different banks
    const int PS = NB + 4;

    // Warp 0: rigid-body transform and the torsion tree.  Torsion k is lane
    // k < 32; its fragment's full transform M_{k+1} = M_0 o L_a o ... o L_k.
    // Teams of several warps (the local search, latency-bound) build it by
    // pointer jumping over the tree: each round composes a lane's partial
    // product with its current ancestor's (shuffles) and jumps to that
    // ancestor's ancestor, so depth d takes ceil(log2 d) + 1 rounds.  One-warp
    // teams go level by level through shared memory (measured faster inside
    // the serving kernel, equal elsewhere).
    if (tm.warp() == 0) {
        __syncwarp();
        float qw = geno[3], qx = geno[4], qy = geno[5], qz = geno[6];
        const float qn2 = qw * qw + qx * qx + qy * qy + qz * qz;
        if (qn2 >= 1e-24f) {
            const float qi = rsqrtf(qn2);
            qw *= qi; qx *= qi; qy *= qi; qz *= qi;
        } else {
            qw = 1.f; qx = qy = qz = 0.f;
        }
        // M_0: the rotation of the normalised quaternion (no translation)
        const float q00 = 1.f - 2.f * (qy * qy + qz * qz), q01 = 2.f * (qx * qy - qw * qz), q02 = 2.f * (qx * qz + qw * qy);
        const float q10 = 2.f * (qx * qy + qw * qz), q11 = 1.f - 2.f * (qx * qx + qz * qz), q12 = 2.f * (qy * qz - qw * qx);
        const float q20 = 2.f * (qx * qz - qw * qy), q21 = 2.f * (qy * qz + qw * qx), q22 = 1.f - 2.f * (qx * qx + qy * qy);
        if (lane == 0) {
            M[0] = make_float4(q00, q01, q02, 0.f);
            M[1] = make_float4(q10, q11, q12, 0.f);
            M[2] = make_float4(q20, q21, q22, 0.f);
        }
        float r00 = 0, r01 = 0, r02 = 0, r10 = 0, r11 = 0, r12 = 0, r20 = 0, r21 = 0, r22 = 0, t0 = 0, t1 = 0, t2 = 0;
        int up = 0;         // fragment the lane's partial product reaches up to (0: the root, done)
        if (lane < T) {
            // reduce to [-pi, pi] (one multiple of 2 pi), then the fast intrinsic
            float tau = geno[ldg(L.tors_gene + lane)];
            tau = fmaf(-6.28318530717958647692f, rintf(tau * 0.15915494309189533577f), tau);
            float s, c;
            __sincosf(tau, &s, &c);
            const float4 u = ldg(L.tors_u + lane), b = ldg(L.tors_b + lane);
            const float oc = 1.f - c;
            r00 = fmaf(oc * u.x, u.x, c);        r01 = fmaf(oc * u.x, u.y, -s * u.z); r02 = fmaf(oc * u.x, u.z, s * u.y);
            r10 = fmaf(oc * u.y, u.x, s * u.z);  r11 = fmaf(oc * u.y, u.y, c);       r12 = fmaf(oc * u.y, u.z, -s * u.x);
            r20 = fmaf(oc * u.z, u.x, -s * u.y); r21 = fmaf(oc * u.z, u.y, s * u.x); r22 = fmaf(oc * u.z, u.z, c);
            t0 = b.x - (r00 * b.x + r01 * b.y + r02 * b.z);
            t1 = b.y - (r10 * b.x + r11 * b.y + r12 * b.z);
            t2 = b.z - (r20 * b.x + r21 * b.y + r22 * b.z);
            up = ldg(L.frag + lane + 1).z;
        }
        // (A o B): rotation R_A R_B, translation R_A t_B + t_A; A = (a.., ta..)
        auto compose = [&](float a00, float a01, float a02, float a10, float a11, float a12, float a20, float a21,
                           float a22, float ta0, float ta1, float ta2) {
            const float n00 = a00 * r00 + a01 * r10 + a02 * r20, n01 = a00 * r01 + a01 * r11 + a02 * r21;
            const float n02 = a00 * r02 + a01 * r12 + a02 * r22;
            const float n10 = a10 * r00 + a11 * r10 + a12 * r20, n11 = a10 * r01 + a11 * r11 + a12 * r21;
            const float n12 = a10 * r02 + a11 * r12 + a12 * r22;
            const float n20 = a20 * r00 + a21 * r10 + a22 * r20, n21 = a20 * r01 + a21 * r11 + a22 * r21;
            const float n22 = a20 * r02 + a21 * r12 + a22 * r22;
            const float m0 = a00 * t0 + a01 * t1 + a02 * t2 + ta0, m1 = a10 * t0 + a11 * t1 + a12 * t2 + ta1;
            const float m2 = a20 * t0 + a21 * t1 + a22 * t2 + ta2;
            r00 = n00; r01 = n01; r02 = n02; r10 = n10; r11 = n11; r12 = n12; r20 = n20; r21 = n21; r22 = n22;
            t0 = m0; t1 = m1; t2 = m2;
        };
        if (W == 1) {
            // level by level: M_{k+1} = M_parent o L_k
            const int depth = lane < T ? ldg(L.frag + lane + 1).w : 0, parent = up;
            for (int d = 1; d <= L.max_depth; ++d) {
                __syncwarp();
                if (lane < T && depth == d) {
                    const float4 p0 = M[3 * parent], p1 = M[3 * parent + 1], p2 = M[3 * parent + 2];
                    float4 *o = M + 3 * (lane + 1);
                    o[0] = make_float4(p0.x * r00 + p0.y * r10 + p0.z * r20, p0.x * r01 + p0.y * r11 + p0.z * r21,
                                       p0.x * r02 + p0.y * r12 + p0.z * r22, p0.x * t0 + p0.y * t1 + p0.z * t2 + p0.w);
                    o[1] = make_float4(p1.x * r00 + p1.y * r10 + p1.z * r20, p1.x * r01 + p1.y * r11 + p1.z * r21,
                                       p1.x * r02 + p1.y * r12 + p1.z * r22, p1.x * t0 + p1.y * t1 + p1.z * t2 + p1.w);
                    o[2] = make_float4(p2.x * r00 + p2.y * r10 + p2.z * r20, p2.x * r01 + p2.y * r11 + p2.z * r21,
                                       p2.x * r02 + p2.y * r12 + p2.z * r22, p2.x * t0 + p2.y * t1 + p2.z * t2 + p2.w);
                }
            }
            (void)compose;
        } else {
            if (lane < T && up == 0) compose(q00, q01, q02, q10, q11, q12, q20, q21, q22, 0.f, 0.f, 0.f);
            // at most 6 rounds: depth <= 32 = 2^5
            for (int jump = 0; jump < 6 && __any_sync(0xffffffffu, lane < T && up != 0); ++jump) {
                const int src = up > 0 ? up - 1 : lane;  // lane holding fragment `up`
                const float a00 = __shfl_sync(0xffffffffu, r00, src), a01 = __shfl_sync(0xffffffffu, r01, src);
                const float a02 = __shfl_sync(0xffffffffu, r02, src), a10 = __shfl_sync(0xffffffffu, r10, src);
                const float a11 = __shfl_sync(0xffffffffu, r11, src), a12 = __shfl_sync(0xffffffffu, r12, src);
                const float a20 = __shfl_sync(0xffffffffu, r20, src), a21 = __shfl_sync(0xffffffffu, r21, src);
                const float a22 = __shfl_sync(0xffffffffu, r22, src), b0 = __shfl_sync(0xffffffffu, t0, src);
                const float b1 = __shfl_sync(0xffffffffu, t1, src), b2 = __shfl_sync(0xffffffffu, t2, src);
                const int up2 = __shfl_sync(0xffffffffu, up, src);
                if (lane < T && up != 0) {
                    compose(a00, a01, a02, a10, a11, a12, a20, a21, a22, b0, b1, b2);
                    up = up2;
                }
            }
            if (lane < T) {
                float4 *o = M + 3 * (lane + 1);
                o[0] = make_float4(r00, r01, r02, t0);
                o[1] = make_float4(r10, r11, r12, t1);
                o[2] = make_float4(r20, r21, r22, t2);
            }
        }
    }
    // Force accumulators start at zero: W = 1 adds pair forces straight into
    // the per-atom forces, W > 1 into per-group partials (zeroed by warps
    // 1.., while warp 0 composes the tree).
    float4 *Fv = reinterpret_cast<float4 *>(ws + Y.f);
    if (GRAD) {
        if (W == 1)
            for (int k = r; k < NB; k += S) Fv[k] = make_float4(0.f, 0.f, 0.f, 0.f);
        else if (r >= 32)
            for (int k = r - 32; k < 4 * W * PS; k += S - 32) PF[k] = make_float4(0.f, 0.f, 0.f, 0.f);
    }
    tm.sync();

    // Atom positions relative to t (padding atoms up to a multiple of 8 at
    // 0).  The thread that places an atom also sends out the reads of its
    // three map cells, staged into shared memory asynchronously: they are in
    // flight through the pair rounds, and the same thread reads them back
    // (consecutive atoms on consecutive lanes).
    const float tux = (geno[0] - G.ox) * G.inv_h, tuy = (geno[1] - G.oy) * G.inv_h, tuz = (geno[2] - G.oz) * G.inv_h;
    float4 *Cst = reinterpret_cast<float4 *>(ws + Y.cst);
    for (int i = r; i < NB; i += S) {
        float4 x = make_float4(0.f, 0.f, 0.f, 0.f);
        if (i < N) {
            const float4 p = ldg(L.ref + i);
            const int meta = ldg(L.meta + i), f = meta >> 8;
            const float4 m0 = M[3 * f], m1 = M[3 * f + 1], m2 = M[3 * f + 2];
            x = make_float4(fmaf(m0.x, p.x, fmaf(m0.y, p.y, fmaf(m0.z, p.z, m0.w))),
                            fmaf(m1.x, p.x, fmaf(m1.y, p.y, fmaf(m1.z, p.z, m1.w))),
                            fmaf(m2.x, p.x, fmaf(m2.y, p.y, fmaf(m2.z, p.z, m2.w))), 0.f);
            atom_stage(G, ldg(G.map_of_type + (meta & 255)), fmaf(x.x, G.inv_h, tux), fmaf(x.y, G.inv_h, tuy),
                       fmaf(x.z, G.inv_h, tuz), Cst + 6 * i);
        }
        float *xp = reinterpret_cast<float *>(XP), *zp = reinterpret_cast<float *>(ZP);
        const int prev = (i & ~7) | ((i + 7) & 7);
        xp[4 * i] = x.x;
        xp[4 * i + 2] = x.y;
        zp[2 * i] = x.z;
        xp[4 * prev + 1] = x.x;
        xp[4 * prev + 3] = x.y;
        zp[2 * prev + 1] = x.z;
    }
    cp_async_commit();
    tm.sync();

    // Intramolecular pairs, systolic: in a step, lane l of group q holds its
    // own atom of block A and, passed one lane along per round, the force
    // owed to the atom of block B it meets; after 8 rounds that force is back
    // at the lane owning the B atom, and both go to the group's partials.
    // Rounds go two at a time in paired FP32 instructions.
    float e = 0.f;
    {
        const SchedDev &SD = L.sched[W == 1 ? 0 : W == 2 ? 1 : W == 4 ? 2 : 3];
        const int w = tm.warp(), q = 4 * w + (lane >> 3), sl = lane & 7, gb = lane & ~7;
        const int nxt = gb | ((sl + 1) & 7);
        float4 *pq = W == 1 ? Fv : PF + q * PS;  // W = 1: the step's groups touch disjoint atoms
        const int s0 = SD.base[w], s1 = s0 + SD.steps[w];
        f32x2 E2 = dup2(0.f);  // energies of even and odd rounds
        // rounds d and d + 1: the pairs (own atom, atoms 8B + (sl + d) mod 8
        // and the next), coefficients from the records at rq; the force owed
        // to the B atom travels one lane on after each round
        auto round2 = [&](f32x2 XA, f32x2 YA, f32x2 ZA, int B, int d, const float4 *rq, f32x2 &AX, f32x2 &AY,
                          f32x2 &AZ, float &bx, float &by, float &bz) {
            const int j = 8 * B + ((sl + d) & 7);
            const float4 pxy = XP[j];
            const float2 pz = ZP[j];
            const f32x2 PX = pk2(pxy.x, pxy.y), PY = pk2(pxy.z, pxy.w), PZ = pk2(pz.x, pz.y);
            const float4 cn4 = ldg(rq), qd4 = ldg(rq + 32);
            const f32x2 C = pk2(cn4.x, cn4.y), N = pk2(cn4.z, cn4.w), Q = pk2(qd4.x, qd4.y), D = pk2(qd4.z, qd4.w);
            const f32x2 DX = sub2(XA, PX), DY = sub2(YA, PY), DZ = sub2(ZA, PZ);
            const f32x2 R2 = fma2(DX, DX, fma2(DY, DY, mul2(DZ, DZ)));
            const float r2a = R2.x, r2b = R2.y;
            // every round computes; the cutoff selects (one basic block for
            // all rounds, so they overlap)
            float sa = 0.f, sb = 0.f;
            const f32x2 EP = pair_energy2<GRAD>(r2a, r2b, C, N, Q, D, sa, sb);
            const float ea = EP.x, eb = EP.y;
            const bool ina = r2a < kCut2, inb = r2b < kCut2;
            E2 = add2(E2, pk2(ina ? ea : 0.f, inb ? eb : 0.f));
            if (GRAD) {
                // force s d on the own atom, -s d on the partner (fused)
                const float s0 = ina ? sa : 0.f, s1 = inb ? sb : 0.f;
                const f32x2 S2 = pk2(s0, s1);
                AX = fma2(S2, DX, AX);
                AY = fma2(S2, DY, AY);
                AZ = fma2(S2, DZ, AZ);
                bx = __shfl_sync(0xffffffffu, fmaf(-s0, DX.x, bx), nxt);
                by = __shfl_sync(0xffffffffu, fmaf(-s0, DY.x, by), nxt);
                bz = __shfl_sync(0xffffffffu, fmaf(-s0, DZ.x, bz), nxt);
                bx = __shfl_sync(0xffffffffu, fmaf(-s1, DX.y, bx), nxt);
                by = __shfl_sync(0xffffffffu, fmaf(-s1, DY.y, by), nxt);
                bz = __shfl_sync(0xffffffffu, fmaf(-s1, DZ.y, bz), nxt);
            }
        };
        for (int st = s0; st < s1; ++st) {
            const uint32_t ctl = ldg(SD.ctrl + 4 * st + (lane >> 3));
            const int A = SCH_A(ctl), B = SCH_B(ctl);
            const float3 xa = pos(8 * A + sl);
            const f32x2 XA = dup2(xa.x), YA = dup2(xa.y), ZA = dup2(xa.z);
            // records of round pair p: rec[st][p][0][lane] = (c12, c12', cn,
            // cn'), rec[st][p][1][lane] = (qq, qq', ds, ds')
            const float4 *rp = SD.rec + 256 * (size_t)st + lane;
            f32x2 AX = dup2(0.f), AY = dup2(0.f), AZ = dup2(0.f);
            float bx = 0.f, by = 0.f, bz = 0.f;
            if (W == 1 && (ctl & SCH_HALF)) {
                // diagonal blocks, rounds 1-4: the travelling force ends 4
                // lanes on; the atom's owner fetches it from lane sl + 3
                round2(XA, YA, ZA, B, 1, rp, AX, AY, AZ, bx, by, bz);
                round2(XA, YA, ZA, B, 3, rp + 64, AX, AY, AZ, bx, by, bz);
                if (GRAD) {
                    const int src = gb | ((sl + 3) & 7);
                    bx = __shfl_sync(0xffffffffu, bx, src);
                    by = __shfl_sync(0xffffffffu, by, src);
                    bz = __shfl_sync(0xffffffffu, bz, src);
                }
            } else {
#pragma unroll
                for (int p = 0; p < 4; ++p) round2(XA, YA, ZA, B, 2 * p, rp + 64 * p, AX, AY, AZ, bx, by, bz);
            }
            if (GRAD && (ctl & SCH_VALID)) {
                float4 pa = pq[8 * A + sl];
                pa.x += AX.x + AX.y;
                pa.y += AY.x + AY.y;
                pa.z += AZ.x + AZ.y;
                pq[8 * A + sl] = pa;  // (a diagonal block's second update below is this thread's too)
                float4 pb = pq[8 * B + sl];
                pb.x += bx; pb.y += by; pb.z += bz;
                pq[8 * B + sl] = pb;
            }
            // W = 1: the next step may give these atoms to another group
            if (GRAD && W == 1) __syncwarp();
        }
        e = E2.x + E2.y;
    }
    // pair forces complete: W = 1 in Fv, W > 1 in every group's partials
    if (GRAD) tm.sync();
    cp_async_wait_all();

    // Per atom: grid energy and force from the staged cells, the complete
    // force (W = 1: the pair force in Fv plus the grid part; W > 1: the grid
    // part plus the partial rows of the groups whose steps touched the atom's
    // block, ascending group order) and the torque (x_i - t) x f_i.
    // W = 1 keeps the torques (and below the fragment sums) in the staged-cell
    // area: atom i's torque goes to its own first cell slot, written by the
    // thread that has just read that atom's cells
    float4 *Tq = W == 1 ? Cst : reinterpret_cast<float4 *>(ws + Y.tq);
    constexpr int TS = W == 1 ? 6 : 1;  // float4 stride of the torques
    const uint32_t *gmask = L.sched[W == 1 ? 0 : W == 2 ? 1 : W == 4 ? 2 : 3].gmask;
    for (int i = r; i < N; i += S) {
        const float3 xi = pos(i);
        AtomCells A0;
        atom_unstage(G, ldg(L.ref + i).w, fmaf(xi.x, G.inv_h, tux), fmaf(xi.y, G.inv_h, tuy),
                     fmaf(xi.z, G.inv_h, tuz), Cst + 6 * i, A0);
        float3 g;
        e += atom_grid_energy<GRAD>(G, A0, g);
        if (GRAD) {
            float fx, fy, fz;
            if (W == 1) {
                const float4 pf = Fv[i];
                fx = pf.x + g.x; fy = pf.y + g.y; fz = pf.z + g.z;
            } else {
                const uint32_t m = ldg(gmask + (i >> 3));
                fx = g.x; fy = g.y; fz = g.z;
#pragma unroll
                for (int q = 0; q < 4 * W; ++q)
                    if (m & (1u << q)) {
                        const float4 v = PF[q * PS + i];
                        fx += v.x; fy += v.y; fz += v.z;
                    }
            }
            Fv[i] = make_float4(fx, fy, fz, 0.f);
            Tq[TS * i] = make_float4(xi.y * fz - xi.z * fy, xi.z * fx - xi.x * fz, xi.x * fy - xi.y * fx, 0.f);
        }
    }
    if (!GRAD) return team_sum(tm, e, red);
    // the energy's warp partials go out now, off the critical path; the team
    // adds them after the gradient's barrier (their slots are rewritten only
    // after the next evaluation's first barrier)
    const float ew = warp_sum(e);
    if (W > 1 && lane == 0) red[16 + tm.warp()] = ew;
    tm.sync();

    // Gradient.  W = 1: per-fragment sums first, then torsion k sums the
    // fragments it moves (a contiguous run in depth-first order).  W > 1:
    // torsion k sums its contiguous atom range directly.  Range T is the
    // whole ligand (translation and rotation).  m lanes per range, butterfly.
    // W = 1: fragment f's sums in slots 6f + 1 and 6f + 2 of the staged-cell
    // area (dead once every atom's grid term is done; the torques hold slot 0)
    float4 *FS = Cst + 1;
    const int F = L.n_frag;
    if (W == 1) {
        const int ml = lanes_log2(F, S, 32), m = 1 << ml, sub = r & (m - 1);
        for (int b0 = 0; b0 < F; b0 += (S >> ml)) {
            const int f = b0 + (r >> ml);
            const bool act = f < F;
            int lo = 0, hi = 0;
            if (act) {
                const int4 fr = ldg(L.frag + f);
                lo = fr.x;
                hi = fr.y;
            }
            float a0 = 0, a1 = 0, a2 = 0, a3 = 0, a4 = 0, a5 = 0;
            for (int i = lo + sub; i < hi; i += m) {
                const float4 fv = Fv[i], t = Tq[TS * i];
                a0 += fv.x; a1 += fv.y; a2 += fv.z;
                a3 += t.x; a4 += t.y; a5 += t.z;
            }
            group_sum6(a0, a1, a2, a3, a4, a5, ml);
            if (act && sub == 0) {
                FS[6 * f] = make_float4(a0, a1, a2, 0.f);
                FS[6 * f + 1] = make_float4(a3, a4, a5, 0.f);
            }
        }
        tm.sync();
    }
    float *grad = ws + Y.grad;
    {
        const int R = T + 1, ml = lanes_log2(R, S, 32), m = 1 << ml, sub = r & (m - 1);
        for (int b0 = 0; b0 < R; b0 += (S >> ml)) {
            const int k = b0 + ((lane >> ml) * W + tm.warp());
            const bool act = k < R;
            int lo = 0, hi = 0;
            if (act) {
                if (W == 1) {
                    lo = k < T ? k + 1 : 0;
                    hi = k < T ? ldg(L.sub_end + k + 1) : F;
                } else if (k < T) {
                    const int2 rg = ldg(L.tors_range + k);
                    lo = rg.x;
                    hi = rg.y;
                } else {
                    hi = N;
                }
            }
            float a0 = 0, a1 = 0, a2 = 0, a3 = 0, a4 = 0, a5 = 0;
#pragma unroll 4
            for (int j = lo + sub; j < hi; j += m) {
                const float4 u = W == 1 ? FS[6 * j] : Fv[j], v = W == 1 ? FS[6 * j + 1] : Tq[TS * j];
                a0 += u.x; a1 += u.y; a2 += u.z;
                a3 += v.x; a4 += v.y; a5 += v.z;
            }
            group_sum6(a0, a1, a2, a3, a4, a5, ml);
            if (act && sub == 0) {
                if (k < T) {  // u_k . sum over the moved atoms of (x_i - x_b) x f_i
                    const int2 ab = ldg(L.tors_ab + k);
                    const float3 xa = pos(ab.x), xb = pos(ab.y);
                    float ux = xb.x - xa.x, uy = xb.y - xa.y, uz = xb.z - xa.z;
                    const float il = rsqrtf(fmaf(ux, ux, fmaf(uy, uy, uz * uz)));
                    ux *= il; uy *= il; uz *= il;
                    const float cx = a3 - (xb.y * a2 - xb.z * a1);
                    const float cy = a4 - (xb.z * a0 - xb.x * a2);
                    const float cz = a5 - (xb.x * a1 - xb.y * a0);
                    grad[ldg(L.tors_gene + k)] = fmaf(ux, cx, fmaf(uy, cy, uz * cz));
                } else {  // dE/dt = sum f; dE/dq = 2 ((0, G) (x) qhat) / |q|, G = torque about t
                    float qw = geno[3], qx = geno[4], qy = geno[5], qz = geno[6];
                    const float qn2 = qw * qw + qx * qx + qy * qy + qz * qz;
                    float qinv = 0.f;
                    if (qn2 >= 1e-24f) {
                        qinv = rsqrtf(qn2);
                        qw *= qinv; qx *= qinv; qy *= qinv; qz *= qinv;
                    } else {
                        qw = 1.f; qx = qy = qz = 0.f;
                    }
                    grad[0] = a0; grad[1] = a1; grad[2] = a2;
                    const float k2 = 2.f * qinv;
                    grad[3] = k2 * (-a3 * qx - a4 * qy - a5 * qz);
                    grad[4] = k2 * (a3 * qw + a4 * qz - a5 * qy);
                    grad[5] = k2 * (-a3 * qz + a4 * qw + a5 * qx);
                    grad[6] = k2 * (a3 * qy - a4 * qx + a5 * qw);
                }
            }
        }
    }
    if (W == 1) {
        __syncwarp();  // publishes grad[]
        return ew;
    }
    tm.sync();  // publishes grad[] and the energy partials
    float et = red[16];
#pragma unroll
    for (int w = 1; w < W; ++w) et += red[16 + w];
    return et;
}

}  // namespace dev
