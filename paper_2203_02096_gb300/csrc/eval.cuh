// eval.cuh -- one warp evaluates the energy (and gradient) of one genotype.
//
// Steps (paper, Section II-A / IV-B): genotype -> pose by rotations along
// the torsion tree; particle-grid energy by trilinear reads of the receptor
// maps; intramolecular pair energy (vdW / H-bond, screened Coulomb,
// desolvation); then the analytic genotype gradient.
//
// GB300 layout: the warp keeps its pose, forces and per-pair force scalars
// in shared memory; ligand constants come through L1 (read-only path);
// each atom-map read is one 32-byte sector of the cell-major grid copy,
// L2-resident.  Every reduction has a fixed order (lane-strided partial sums,
// then an xor butterfly), so results are bit-reproducible run to run.
#pragma once

#include "internal.h"

namespace dev {

constexpr float kDielA = -8.5525f;
constexpr float kDielB = (float)(78.4 + 8.5525);
constexpr float kDielK = 7.7839f;
constexpr float kDielLB = (float)(0.003627 * (78.4 + 8.5525));
constexpr float kDielDeps = (float)((78.4 + 8.5525) * 7.7839 * 0.003627 * (78.4 + 8.5525));
constexpr float kHalfInvSig2 = (float)(1.0 / (2.0 * 3.6 * 3.6));
constexpr float kInvSig2 = (float)(1.0 / (3.6 * 3.6));
constexpr float kCut2 = 64.0f;
constexpr float kFloor2 = 0.25f;
constexpr float kKout = 10.0f;

template <typename T>
__device__ __forceinline__ T ldg(const T *p) { return __ldg(p); }

// Where an atom sits in the grid: cell index, in-cell fractions, clamping
// and the out-of-box penalty (energy and its gradient in kcal/mol/A).
struct CellPos {
    int cell;
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
    c.cell = (iz * (G.ny - 1) + iy) * (G.nx - 1) + ix;
}

// Trilinear read of map m in the located cell; derivatives are with respect
// to the in-cell fractions.
template <bool GRAD>
__device__ __forceinline__ float read_map(const GridDev &G, const CellPos &c, int m, float &gx, float &gy, float &gz) {
    const float4 *p = G.cells + 2 * ((size_t)c.cell * G.M + m);
    const float4 a = ldg(p), b = ldg(p + 1);
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

// Energy of one atom (type map + q * electrostatic + |q| * desolvation +
// out-of-box penalty) and dE/dx.
template <bool GRAD>
__device__ __forceinline__ float atom_grid_energy(const GridDev &G, int map_t, float q, float ux, float uy, float uz,
                                                  float3 &g) {
    CellPos c;
    locate(G, ux, uy, uz, c);
    float tx, ty, tz, ex, ey, ez, dx, dy, dz;
    const float aq = fabsf(q);
    const float vt = read_map<GRAD>(G, c, map_t, tx, ty, tz);
    const float ve = read_map<GRAD>(G, c, G.emap, ex, ey, ez);
    const float vd = read_map<GRAD>(G, c, G.dmap, dx, dy, dz);
    if (GRAD) {
        const float sx = c.cx ? 0.f : G.inv_h, sy = c.cy ? 0.f : G.inv_h, sz = c.cz ? 0.f : G.inv_h;
        g.x = fmaf(sx, fmaf(aq, dx, fmaf(q, ex, tx)), c.gpx);
        g.y = fmaf(sy, fmaf(aq, dy, fmaf(q, ey, ty)), c.gpy);
        g.z = fmaf(sz, fmaf(aq, dz, fmaf(q, ez, tz)), c.gpz);
    }
    return fmaf(aq, vd, fmaf(q, ve, vt)) + c.pen;
}

// Intramolecular pair: energy, and s = (dE/dr)/r (0 below the floor), for
// squared distance r2 < 64.
template <bool GRAD>
__device__ __forceinline__ float pair_energy(float r2, float4 c, float ds, float &s) {
    const float r2e = fmaxf(r2, kFloor2);
    const float rinv = rsqrtf(r2e);
    const float r = r2e * rinv;
    const float ri2 = rinv * rinv, ri6 = ri2 * ri2 * ri2, ri10 = ri6 * ri2 * ri2, ri12 = ri6 * ri6;
    const float ev = c.x * ri12 - c.y * ri6 - c.z * ri10;
    const float ex = __expf(-kDielLB * r);
    const float den = fmaf(kDielK, ex, 1.f);
    const float eps = kDielA + __fdividef(kDielB, den);
    const float eel = c.w * __fdividef(rinv, eps);
    const float eds = ds * __expf(-r2e * kHalfInvSig2);
    if (GRAD) {
        if (r2 >= kFloor2) {
            const float dv = (-12.f * c.x * ri12 + 6.f * c.y * ri6 + 10.f * c.z * ri10) * rinv;
            const float deps = __fdividef(kDielDeps * ex, den * den);
            const float del = -eel * __fdividef(fmaf(r, deps, eps), eps * r);
            const float dds = -eds * r * kInvSig2;
            s = (dv + del + dds) * rinv;
        } else {
            s = 0.f;
        }
    }
    return ev + eel + eds;
}

__device__ __forceinline__ float warp_sum(float v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// Evaluates the genotype stored at ws[W.geno ...]; returns E on every lane.
// With GRAD, dE/dgenotype is left at ws[W.grad ...].
template <bool GRAD>
__device__ float eval_warp(const LigandDev &L, const GridDev &G, float *ws, const WarpLayout &W, const int lane) {
    const float *geno = ws + W.geno;
    float4 *M = reinterpret_cast<float4 *>(ws + W.M);
    float4 *X = reinterpret_cast<float4 *>(ws + W.x);
    const int T = L.n_tors, N = L.n_atoms, P = L.n_pairs;

    // Rigid-body part: positions are kept relative to the translation t.
    const float tx = geno[0], ty = geno[1], tz = geno[2];
    float qw = geno[3], qx = geno[4], qy = geno[5], qz = geno[6];
    const float qn2 = qw * qw + qx * qx + qy * qy + qz * qz;
    float qinv = 0.f;
    if (qn2 >= 1e-24f) {
        qinv = rsqrtf(qn2);
        qw *= qinv; qx *= qinv; qy *= qinv; qz *= qinv;
    } else {
        qw = 1.f; qx = qy = qz = 0.f;
    }
    if (lane == 0) {
        M[0] = make_float4(1.f - 2.f * (qy * qy + qz * qz), 2.f * (qx * qy - qw * qz), 2.f * (qx * qz + qw * qy), 0.f);
        M[1] = make_float4(2.f * (qx * qy + qw * qz), 1.f - 2.f * (qx * qx + qz * qz), 2.f * (qy * qz - qw * qx), 0.f);
        M[2] = make_float4(2.f * (qx * qz - qw * qy), 2.f * (qy * qz + qw * qx), 1.f - 2.f * (qx * qx + qy * qy), 0.f);
    }
    // Lane k holds the local transform of torsion k: rotation by tau_k about
    // the reference bond axis through atom b (Rodrigues, right-hand rule).
    float r00 = 0, r01 = 0, r02 = 0, r10 = 0, r11 = 0, r12 = 0, r20 = 0, r21 = 0, r22 = 0, t0 = 0, t1 = 0, t2 = 0;
    int depth = 0, parent = 0;
    if (lane < T) {
        float s, c;
        sincosf(geno[ldg(L.tors_gene + lane)], &s, &c);
        const float4 u = ldg(L.tors_u + lane), b = ldg(L.tors_b + lane);
        const float oc = 1.f - c;
        r00 = fmaf(oc * u.x, u.x, c);       r01 = fmaf(oc * u.x, u.y, -s * u.z); r02 = fmaf(oc * u.x, u.z, s * u.y);
        r10 = fmaf(oc * u.y, u.x, s * u.z); r11 = fmaf(oc * u.y, u.y, c);       r12 = fmaf(oc * u.y, u.z, -s * u.x);
        r20 = fmaf(oc * u.z, u.x, -s * u.y); r21 = fmaf(oc * u.z, u.y, s * u.x); r22 = fmaf(oc * u.z, u.z, c);
        t0 = b.x - (r00 * b.x + r01 * b.y + r02 * b.z);
        t1 = b.y - (r10 * b.x + r11 * b.y + r12 * b.z);
        t2 = b.z - (r20 * b.x + r21 * b.y + r22 * b.z);
        const int4 fr = ldg(L.frag + lane + 1);
        parent = fr.z;
        depth = fr.w;
    }
    // Forward kinematics, one tree level at a time: M_child = M_parent o L_k.
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
    __syncwarp();

    // Atoms: position, then the particle-grid term.
    const float tux = (tx - G.ox) * G.inv_h, tuy = (ty - G.oy) * G.inv_h, tuz = (tz - G.oz) * G.inv_h;
    float4 *Fv = reinterpret_cast<float4 *>(ws + W.f);
    float e = 0.f;
    for (int i = lane; i < N; i += DOCK_WARP) {
        const float4 p = ldg(L.ref + i);
        const int meta = ldg(L.meta + i);
        const int f = meta >> 8;
        const float4 m0 = M[3 * f], m1 = M[3 * f + 1], m2 = M[3 * f + 2];
        const float dx = fmaf(m0.x, p.x, fmaf(m0.y, p.y, fmaf(m0.z, p.z, m0.w)));
        const float dy = fmaf(m1.x, p.x, fmaf(m1.y, p.y, fmaf(m1.z, p.z, m1.w)));
        const float dz = fmaf(m2.x, p.x, fmaf(m2.y, p.y, fmaf(m2.z, p.z, m2.w)));
        X[i] = make_float4(dx, dy, dz, 0.f);
        float3 g;
        e += atom_grid_energy<GRAD>(G, ldg(G.map_of_type + (meta & 255)), p.w, fmaf(dx, G.inv_h, tux),
                                    fmaf(dy, G.inv_h, tuy), fmaf(dz, G.inv_h, tuz), g);
        if (GRAD) Fv[i] = make_float4(g.x, g.y, g.z, 0.f);
    }
    __syncwarp();

    // Intramolecular pairs, lane-strided; s_p = (dE/dr)/r kept per pair.
    float *S = ws + W.s;
    for (int p = lane; p < P; p += DOCK_WARP) {
        const uint32_t ij = ldg(L.pair_ij + p);
        const float4 xi = X[ij & 0xffffu], xj = X[ij >> 16];
        const float ddx = xi.x - xj.x, ddy = xi.y - xj.y, ddz = xi.z - xj.z;
        const float r2 = fmaf(ddx, ddx, fmaf(ddy, ddy, ddz * ddz));
        float s = 0.f;
        if (r2 < kCut2) e += pair_energy<GRAD>(r2, ldg(L.pair_c + p), ldg(L.pair_ds + p), s);
        if (GRAD) S[p] = s;
    }
    e = warp_sum(e);
    if (!GRAD) return e;
    __syncwarp();

    // Forces: dE/dx_i += s_p (x_i - x_partner) over the atom's pairs, in CSR order.
    for (int i = lane; i < N; i += DOCK_WARP) {
        const float4 xi = X[i];
        float4 fi = Fv[i];
        const int e0 = ldg(L.adj_off + i), e1 = ldg(L.adj_off + i + 1);
        for (int k = e0; k < e1; ++k) {
            const uint32_t a = ldg(L.adj + k);
            const float s = S[a & 0xffffu];
            const float4 xo = X[a >> 16];
            fi.x = fmaf(s, xi.x - xo.x, fi.x);
            fi.y = fmaf(s, xi.y - xo.y, fi.y);
            fi.z = fmaf(s, xi.z - xo.z, fi.z);
        }
        Fv[i] = fi;
    }
    __syncwarp();

    // Per-fragment sums of f_i and (x_i - t) x f_i.
    float4 *FS = reinterpret_cast<float4 *>(ws + W.fs);
    for (int f = lane; f < L.n_frag; f += DOCK_WARP) {
        const int4 fr = ldg(L.frag + f);
        float fx = 0, fy = 0, fz = 0, gx = 0, gy = 0, gz = 0;
        for (int i = fr.x; i < fr.y; ++i) {
            const float4 xi = X[i], fi = Fv[i];
            fx += fi.x; fy += fi.y; fz += fi.z;
            gx += xi.y * fi.z - xi.z * fi.y;
            gy += xi.z * fi.x - xi.x * fi.z;
            gz += xi.x * fi.y - xi.y * fi.x;
        }
        FS[2 * f] = make_float4(fx, fy, fz, 0.f);
        FS[2 * f + 1] = make_float4(gx, gy, gz, 0.f);
    }
    __syncwarp();

    float *grad = ws + W.grad;
    // Torsion k: u_k . sum over its subtree of (x_i - x_b) x f_i.
    if (lane < T) {
        const int f0 = lane + 1, f1 = ldg(L.sub_end + f0);
        float fx = 0, fy = 0, fz = 0, gx = 0, gy = 0, gz = 0;
        for (int f = f0; f < f1; ++f) {
            const float4 a = FS[2 * f], b = FS[2 * f + 1];
            fx += a.x; fy += a.y; fz += a.z;
            gx += b.x; gy += b.y; gz += b.z;
        }
        const int2 ab = ldg(L.tors_ab + lane);
        const float4 xa = X[ab.x], xb = X[ab.y];
        float ux = xb.x - xa.x, uy = xb.y - xa.y, uz = xb.z - xa.z;
        const float il = rsqrtf(fmaf(ux, ux, fmaf(uy, uy, uz * uz)));
        ux *= il; uy *= il; uz *= il;
        const float cx = gx - (xb.y * fz - xb.z * fy);
        const float cy = gy - (xb.z * fx - xb.x * fz);
        const float cz = gz - (xb.x * fy - xb.y * fx);
        grad[ldg(L.tors_gene + lane)] = fmaf(ux, cx, fmaf(uy, cy, uz * cz));
    }
    // Whole-ligand force and torque about t, fixed-order butterfly.
    float a0 = 0, a1 = 0, a2 = 0, a3 = 0, a4 = 0, a5 = 0;
    for (int f = lane; f < L.n_frag; f += DOCK_WARP) {
        const float4 a = FS[2 * f], b = FS[2 * f + 1];
        a0 += a.x; a1 += a.y; a2 += a.z; a3 += b.x; a4 += b.y; a5 += b.z;
    }
    a0 = warp_sum(a0); a1 = warp_sum(a1); a2 = warp_sum(a2);
    a3 = warp_sum(a3); a4 = warp_sum(a4); a5 = warp_sum(a5);
    if (lane == 0) {
        grad[0] = a0; grad[1] = a1; grad[2] = a2;
        // dE/dq = 2 ((0, G) (x) qhat) / |q|
        const float k2 = 2.f * qinv;
        grad[3] = k2 * (-a3 * qx - a4 * qy - a5 * qz);
        grad[4] = k2 * (a3 * qw + a4 * qz - a5 * qy);
        grad[5] = k2 * (-a3 * qz + a4 * qw + a5 * qx);
        grad[6] = k2 * (a3 * qy - a4 * qx + a5 * qw);
    }
    __syncwarp();
    return e;
}

}  // namespace dev
