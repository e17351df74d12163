// rescore.cuh -- FP64 re-score of final poses: one thread per genotype,
// the energy written out serially in double (same forms and constants as the
// FP32 evaluator).
#pragma once

#include "internal.h"

namespace {

__device__ double interp64(const GridDev &G, int m, const double *u, double &pen) {
    const int n[3] = {G.nx, G.ny, G.nz};
    int i0[3];
    double f[3];
    for (int a = 0; a < 3; ++a) {
        double v = u[a], d = 0.0;
        if (v < 0.0) { d = v; v = 0.0; }
        else if (v > n[a] - 1) { d = v - (n[a] - 1); v = n[a] - 1; }
        int k = (int)floor(v);
        if (k > n[a] - 2) k = n[a] - 2;
        i0[a] = k;
        f[a] = v - k;
        const double dh = d * G.h64;
        pen += 10.0 * dh * dh;
    }
    const long long q = (size_t)m * G.mstride + ((long long)i0[1] * (G.nx - 1) + i0[0]) * G.nz + i0[2];
    const float4 a = G.cells[q], b = G.cells[q + 1];
    const double v[8] = {a.x, a.y, a.z, a.w, b.x, b.y, b.z, b.w};
    double s = 0.0;
    for (int c = 0; c < 8; ++c) {
        const double wx = (c & 1) ? f[0] : 1.0 - f[0];
        const double wy = (c & 2) ? f[1] : 1.0 - f[1];
        const double wz = (c & 4) ? f[2] : 1.0 - f[2];
        s += wx * wy * wz * v[c];
    }
    return s;
}

// FP64 energy of one genotype, written out serially by one thread.
__device__ double rescore64_one(const LigandDev &L, const GridDev &G, const float *__restrict__ g) {
    double M[DOCK_MAX_TORSIONS + 1][12];
    double qw = g[3], qx = g[4], qy = g[5], qz = g[6];
    const double qn = sqrt(qw * qw + qx * qx + qy * qy + qz * qz);
    if (qn >= 1e-12) { qw /= qn; qx /= qn; qy /= qn; qz /= qn; }
    else { qw = 1; qx = qy = qz = 0; }
    const double R0[12] = {1 - 2 * (qy * qy + qz * qz), 2 * (qx * qy - qw * qz), 2 * (qx * qz + qw * qy), 0,
                           2 * (qx * qy + qw * qz), 1 - 2 * (qx * qx + qz * qz), 2 * (qy * qz - qw * qx), 0,
                           2 * (qx * qz - qw * qy), 2 * (qy * qz + qw * qx), 1 - 2 * (qx * qx + qy * qy), 0};
    for (int k = 0; k < 12; ++k) M[0][k] = R0[k];
    // fragments are in depth-first preorder: a parent precedes its children
    for (int f = 1; f < L.n_frag; ++f) {
        const int k = f - 1;
        const int2 ab = L.tors_ab[k];
        const double *pa = L.ref64 + 3 * ab.x, *pb = L.ref64 + 3 * ab.y;
        double u[3] = {pb[0] - pa[0], pb[1] - pa[1], pb[2] - pa[2]};
        const double il = 1.0 / sqrt(u[0] * u[0] + u[1] * u[1] + u[2] * u[2]);
        u[0] *= il; u[1] *= il; u[2] *= il;
        double s, c;
        sincos((double)g[L.tors_gene[k]], &s, &c);
        const double oc = 1 - c;
        const double r[9] = {c + oc * u[0] * u[0],        oc * u[0] * u[1] - s * u[2], oc * u[0] * u[2] + s * u[1],
                             oc * u[1] * u[0] + s * u[2], c + oc * u[1] * u[1],        oc * u[1] * u[2] - s * u[0],
                             oc * u[2] * u[0] - s * u[1], oc * u[2] * u[1] + s * u[0], c + oc * u[2] * u[2]};
        const double t[3] = {pb[0] - (r[0] * pb[0] + r[1] * pb[1] + r[2] * pb[2]),
                             pb[1] - (r[3] * pb[0] + r[4] * pb[1] + r[5] * pb[2]),
                             pb[2] - (r[6] * pb[0] + r[7] * pb[1] + r[8] * pb[2])};
        const double *P = M[L.frag[f].z];
        for (int row = 0; row < 3; ++row) {
            const double *pr = P + 4 * row;
            M[f][4 * row + 0] = pr[0] * r[0] + pr[1] * r[3] + pr[2] * r[6];
            M[f][4 * row + 1] = pr[0] * r[1] + pr[1] * r[4] + pr[2] * r[7];
            M[f][4 * row + 2] = pr[0] * r[2] + pr[1] * r[5] + pr[2] * r[8];
            M[f][4 * row + 3] = pr[0] * t[0] + pr[1] * t[1] + pr[2] * t[2] + pr[3];
        }
    }
    double X[DOCK_MAX_ATOMS][3];
    double e = 0.0;
    for (int i = 0; i < L.n_atoms; ++i) {
        const double *p = L.ref64 + 3 * i;
        const int meta = L.meta[i];
        const double *m = M[meta >> 8];
        double u[3];
        for (int a = 0; a < 3; ++a) {
            X[i][a] = m[4 * a] * p[0] + m[4 * a + 1] * p[1] + m[4 * a + 2] * p[2] + m[4 * a + 3] + (double)g[a];
        }
        u[0] = (X[i][0] - G.ox64) / G.h64;
        u[1] = (X[i][1] - G.oy64) / G.h64;
        u[2] = (X[i][2] - G.oz64) / G.h64;
        const double q = L.q64[i];
        double pen = 0.0, dummy = 0.0;
        e += interp64(G, G.map_of_type[meta & 255], u, pen) + q * interp64(G, G.emap, u, dummy) +
             fabs(q) * interp64(G, G.dmap, u, dummy) + pen;
    }
    const double lb = 0.003627 * (78.4 + 8.5525);
    for (int p = 0; p < L.n_pairs; ++p) {
        const uint32_t ij = L.pair_ij[p];
        const double *xi = X[ij & 0xffff], *xj = X[ij >> 16];
        const double dx = xi[0] - xj[0], dy = xi[1] - xj[1], dz = xi[2] - xj[2];
        double r = sqrt(dx * dx + dy * dy + dz * dz);
        if (r >= 8.0) continue;
        if (r < 0.5) r = 0.5;
        const double *c = L.pair_c64 + 5 * p;
        const double ri2 = 1.0 / (r * r), ri6 = ri2 * ri2 * ri2;
        const double eps = -8.5525 + (78.4 + 8.5525) / (1.0 + 7.7839 * exp(-lb * r));
        e += c[0] * ri6 * ri6 - c[1] * ri6 - c[2] * ri6 * ri2 * ri2 + c[3] / (eps * r) +
             c[4] * exp(-r * r / (2.0 * 3.6 * 3.6));
    }
    return e;
}

}  // namespace
