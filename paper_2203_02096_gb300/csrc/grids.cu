// grids.cu -- receptor grid maps on the device: the z-column quad copy read
// by the evaluator, and the direct-sum map builder (the "reaction field for the
// protein" of Section II-A computed from receptor atoms).
#include "forcefield.h"
#include "internal.h"

namespace {

// Z-column quad copy: thread per (column, z plane, map), the quad of node
// values (ix, iy), (ix+1, iy), (ix, iy+1), (ix+1, iy+1) -> one float4.
__global__ void relayout_kernel(const float *__restrict__ nodes, int nx, int ny, int nz, int M, float4 *cells) {
    const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const long long ncol = (long long)(nx - 1) * (ny - 1);
    if (idx >= ncol * nz * M) return;
    const int iz = (int)(idx % nz);
    const long long col = (idx / nz) % ncol;
    const int m = (int)(idx / (nz * ncol));
    const int ix = (int)(col % (nx - 1)), iy = (int)(col / (nx - 1));
    const size_t plane = (size_t)nx * ny;
    const float *b = nodes + (size_t)m * plane * nz + (size_t)iz * plane + (size_t)iy * nx + ix;
    cells[idx] = make_float4(b[0], b[1], b[nx], b[nx + 1]);
}

struct MapConst {
    float c12[7][7], c6[7][7], c10[7][7];  // [ligand type][receptor type], weights folded
    float solpar[7], vol[7];
};
__constant__ MapConst kMap;

constexpr int kRecTile = 256;

// Thread per grid node; receptor atoms (xyz relative to the grid origin,
// w = charge) streamed through shared memory.
// Per-term arithmetic in FP32, sums in FP64, type maps capped at +1e5.
__global__ void __launch_bounds__(128)
build_maps_kernel(int n_rec, const float4 *__restrict__ rec, const int *__restrict__ rtype, int nx, int ny, int nz,
                  float h, int n_tmaps, int4 mt_lo, int4 mt_hi, float *nodes) {
    __shared__ float4 s_rec[kRecTile];
    __shared__ int s_t[kRecTile];
    const long long n_nodes = (long long)nx * ny * nz;
    const long long node = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const int ix = (int)(node % nx), iy = (int)((node / nx) % ny), iz = (int)(node / ((long long)nx * ny));
    // receptor coordinates arrive relative to the grid origin; i*h is exact
    const float px = ix * h, py = iy * h, pz = iz * h;
    const int mt[8] = {mt_lo.x, mt_lo.y, mt_lo.z, mt_lo.w, mt_hi.x, mt_hi.y, mt_hi.z, mt_hi.w};
    double acc[9];
    for (int m = 0; m < 9; ++m) acc[m] = 0.0;
    const float lb = (float)(ff::kDielLambda * ff::kDielB);
    const float wel = (float)(ff::kWel * ff::kCoulomb), wds = (float)ff::kWds, qs = (float)ff::kQsolv;
    for (int base = 0; base < n_rec; base += kRecTile) {
        __syncthreads();
        for (int k = threadIdx.x; k < kRecTile && base + k < n_rec; k += blockDim.x) {
            s_rec[k] = rec[base + k];
            s_t[k] = rtype[base + k];
        }
        __syncthreads();
        const int cnt = min(kRecTile, n_rec - base);
        if (node >= n_nodes) continue;
        for (int k = 0; k < cnt; ++k) {
            const float4 a = s_rec[k];
            const int tj = s_t[k];
            const float dx = px - a.x, dy = py - a.y, dz = pz - a.z;
            const float r2 = fmaxf(dx * dx + dy * dy + dz * dz, 0.25f);
            const float rinv = rsqrtf(r2), r = r2 * rinv;
            const float ri2 = rinv * rinv, ri6 = ri2 * ri2 * ri2, ri10 = ri6 * ri2 * ri2, ri12 = ri6 * ri6;
            const float g = __expf(-r2 * (float)(1.0 / (2.0 * ff::kSigma * ff::kSigma)));
            const float vj = kMap.vol[tj];
            const float sj = kMap.solpar[tj] + qs * fabsf(a.w);
            for (int m = 0; m < n_tmaps; ++m) {
                const int t = mt[m];
                const float e = kMap.c12[t][tj] * ri12 - kMap.c6[t][tj] * ri6 - kMap.c10[t][tj] * ri10 +
                                wds * (kMap.solpar[t] * vj + sj * kMap.vol[t]) * g;
                acc[m] += (double)e;
            }
            const float eps = (float)ff::kDielA + __fdividef((float)ff::kDielB, fmaf((float)ff::kDielK, __expf(-lb * r), 1.f));
            acc[n_tmaps] += (double)(wel * a.w * __fdividef(rinv, eps));
            acc[n_tmaps + 1] += (double)(wds * qs * vj * g);
        }
    }
    if (node >= n_nodes) return;
    for (int m = 0; m < n_tmaps + 2; ++m) {
        double v = acc[m];
        if (m < n_tmaps && v > ff::kMapCap) v = ff::kMapCap;
        nodes[(size_t)m * n_nodes + node] = (float)v;
    }
}

}  // namespace

cudaError_t launch_relayout(const GridDev &g, float4 *cells, cudaStream_t s) {
    const long long n = (long long)(g.nx - 1) * (g.ny - 1) * g.nz * g.M;
    relayout_kernel<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(g.nodes, g.nx, g.ny, g.nz, g.M, cells);
    return cudaGetLastError();
}

cudaError_t launch_build_maps(int n_rec, const float4 *rec_rel, const int *rtype, int nx, int ny, int nz, double h,
                              int n_tmaps, const int *map_types, float *nodes, cudaStream_t s) {
    MapConst c{};
    for (int a = 0; a < 7; ++a) {
        c.solpar[a] = (float)ff::kTypes[a].solpar;
        c.vol[a] = (float)ff::kTypes[a].vol;
        for (int b = 0; b < 7; ++b) {
            double c12, c6, c10;
            ff::vdw_coefs(a, b, c12, c6, c10);
            c.c12[a][b] = (float)c12;
            c.c6[a][b] = (float)c6;
            c.c10[a][b] = (float)c10;
        }
    }
    cudaError_t e = cudaMemcpyToSymbolAsync(kMap, &c, sizeof(c), 0, cudaMemcpyHostToDevice, s);
    if (e != cudaSuccess) return e;
    int mt[8] = {0, 0, 0, 0, 0, 0, 0, 0};
    for (int m = 0; m < n_tmaps; ++m) mt[m] = map_types[m];
    const long long n = (long long)nx * ny * nz;
    build_maps_kernel<<<(unsigned)((n + 127) / 128), 128, 0, s>>>(n_rec, rec_rel, rtype, nx, ny, nz, (float)h, n_tmaps,
                                                                    make_int4(mt[0], mt[1], mt[2], mt[3]),
                                                                    make_int4(mt[4], mt[5], mt[6], mt[7]), nodes);
    return cudaGetLastError();
}
