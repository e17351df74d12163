// score.cu -- batched energy / gradient / pose kernels, and the FP64
// re-scoring of final poses.
#include "eval.cuh"

namespace {

constexpr int kScoreWarps = 4;  // warps per block of the batched evaluators

// MINB: blocks per SM the register allocation must leave room for (the
// register cap: 65536 / (128 MINB) registers per thread; 1 = the compiler's
// own choice); chosen per context, see dock_set_option.
template <bool GRAD, int MINB>
__global__ void __launch_bounds__(kScoreWarps * 32, MINB)
score_kernel(LigandDev L, GridDev G, const float *__restrict__ geno, int B, float *__restrict__ E,
             float *__restrict__ grad, EvalLayout W) {
    extern __shared__ float4 smem4[];
    float *ws = reinterpret_cast<float *>(smem4) + (threadIdx.x >> 5) * W.total;
    const int lane = threadIdx.x & 31;
    const dev::Team<1> tm(lane);
    const int nw = gridDim.x * (blockDim.x >> 5);
    const int Gn = L.n_genes;
    for (int b = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); b < B; b += nw) {
        const float *gb = geno + (size_t)b * Gn;
        for (int j = lane; j < Gn; j += 32) ws[W.geno + j] = gb[j];
        __syncwarp();
        const float e = dev::eval_team<1, GRAD>(L, G, ws, W, tm);
        if (lane == 0) E[b] = e;
        if (GRAD)
            for (int j = lane; j < Gn; j += 32) grad[(size_t)b * Gn + j] = ws[W.grad + j];
        __syncwarp();
    }
}

// Pose only: the forward kinematics of the evaluator, written out per atom
// in input order (x = t + d).
__global__ void __launch_bounds__(kScoreWarps * 32)
pose_kernel(LigandDev L, const float *__restrict__ geno, int B, float *__restrict__ xyz, EvalLayout W) {
    extern __shared__ float4 smem4[];
    float *ws = reinterpret_cast<float *>(smem4) + (threadIdx.x >> 5) * W.total;
    const int lane = threadIdx.x & 31;
    const int nw = gridDim.x * (blockDim.x >> 5);
    const int Gn = L.n_genes, T = L.n_tors;
    float4 *M = reinterpret_cast<float4 *>(ws + W.M);
    for (int b = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); b < B; b += nw) {
        const float *g = geno + (size_t)b * Gn;
        float qw = g[3], qx = g[4], qy = g[5], qz = g[6];
        const float qn2 = qw * qw + qx * qx + qy * qy + qz * qz;
        if (qn2 >= 1e-24f) {
            const float qi = rsqrtf(qn2);
            qw *= qi; qx *= qi; qy *= qi; qz *= qi;
        } else {
            qw = 1.f; qx = qy = qz = 0.f;
        }
        if (lane == 0) {
            M[0] = make_float4(1.f - 2.f * (qy * qy + qz * qz), 2.f * (qx * qy - qw * qz), 2.f * (qx * qz + qw * qy), 0.f);
            M[1] = make_float4(2.f * (qx * qy + qw * qz), 1.f - 2.f * (qx * qx + qz * qz), 2.f * (qy * qz - qw * qx), 0.f);
            M[2] = make_float4(2.f * (qx * qz - qw * qy), 2.f * (qy * qz + qw * qx), 1.f - 2.f * (qx * qx + qy * qy), 0.f);
        }
        float r[9] = {0}, t[3] = {0};
        int depth = 0, parent = 0;
        if (lane < T) {
            float s, c;
            sincosf(g[__ldg(L.tors_gene + lane)], &s, &c);
            const float4 u = __ldg(L.tors_u + lane), bb = __ldg(L.tors_b + lane);
            const float oc = 1.f - c;
            r[0] = fmaf(oc * u.x, u.x, c);        r[1] = fmaf(oc * u.x, u.y, -s * u.z); r[2] = fmaf(oc * u.x, u.z, s * u.y);
            r[3] = fmaf(oc * u.y, u.x, s * u.z);  r[4] = fmaf(oc * u.y, u.y, c);        r[5] = fmaf(oc * u.y, u.z, -s * u.x);
            r[6] = fmaf(oc * u.z, u.x, -s * u.y); r[7] = fmaf(oc * u.z, u.y, s * u.x);  r[8] = fmaf(oc * u.z, u.z, c);
            t[0] = bb.x - (r[0] * bb.x + r[1] * bb.y + r[2] * bb.z);
            t[1] = bb.y - (r[3] * bb.x + r[4] * bb.y + r[5] * bb.z);
            t[2] = bb.z - (r[6] * bb.x + r[7] * bb.y + r[8] * bb.z);
            const int4 fr = __ldg(L.frag + lane + 1);
            parent = fr.z;
            depth = fr.w;
        }
        for (int d = 1; d <= L.max_depth; ++d) {
            __syncwarp();
            if (lane < T && depth == d) {
                for (int row = 0; row < 3; ++row) {
                    const float4 p = M[3 * parent + row];
                    M[3 * (lane + 1) + row] =
                        make_float4(p.x * r[0] + p.y * r[3] + p.z * r[6], p.x * r[1] + p.y * r[4] + p.z * r[7],
                                    p.x * r[2] + p.y * r[5] + p.z * r[8], p.x * t[0] + p.y * t[1] + p.z * t[2] + p.w);
                }
            }
        }
        __syncwarp();
        for (int i = lane; i < L.n_atoms; i += 32) {
            const float4 p = __ldg(L.ref + i);
            const int f = __ldg(L.meta + i) >> 8;
            const float4 m0 = M[3 * f], m1 = M[3 * f + 1], m2 = M[3 * f + 2];
            float *o = xyz + ((size_t)b * L.n_atoms + __ldg(L.perm + i)) * 3;
            o[0] = g[0] + fmaf(m0.x, p.x, fmaf(m0.y, p.y, fmaf(m0.z, p.z, m0.w)));
            o[1] = g[1] + fmaf(m1.x, p.x, fmaf(m1.y, p.y, fmaf(m1.z, p.z, m1.w)));
            o[2] = g[2] + fmaf(m2.x, p.x, fmaf(m2.y, p.y, fmaf(m2.z, p.z, m2.w)));
        }
        __syncwarp();
    }
}

template <typename K>
cudaError_t launch_warps(dock_ctx *ctx, K kernel, int B, int wpb, size_t smem, cudaStream_t s, const char *name,
                         void **args) {
    if (B <= 0) return cudaSuccess;
    if (smem > 48 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
    }
    int per_sm = 0;
    cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, wpb * 32, smem);
    if (e != cudaSuccess) return e;
    if (per_sm < 1) return cudaErrorInvalidConfiguration;
    const int need = (B + wpb - 1) / wpb;
    const int cap = per_sm * ctx->num_sms;
    const int blocks = need < cap ? need : cap;
    TimedLaunch tl;
    timing_begin(ctx, kernel_id(ctx, name), s, &tl);
    e = cudaLaunchKernel((const void *)kernel, dim3(blocks), dim3(wpb * 32), args, smem, s);
    timing_end(ctx, s, &tl);
    ++ctx->launches;
    return e;
}

// Warps per block: four when their scratch fits in shared memory, else fewer.
int pick_warps(dock_ctx *ctx, const EvalLayout &W) {
    for (int w = kScoreWarps; w > 1; w >>= 1)
        if (evaluator_smem_ok(ctx, W, w)) return w;
    return 1;
}

}  // namespace

cudaError_t launch_score(dock_ctx *ctx, const LigandDev &L, const GridDev &G, const float *geno, int B, float *E,
                         float *grad, cudaStream_t s) {
    const bool g = grad != nullptr;
    EvalLayout W = eval_layout(L.n_atoms, L.n_frag, L.nb8, g, 1);
    const int wpb = pick_warps(ctx, W);
    const size_t smem = (size_t)W.total * sizeof(float) * wpb;
    LigandDev l = L;
    GridDev gg = G;
    const float *gp = geno;
    float *ep = E, *grp = grad;
    void *args[] = {&l, &gg, &gp, &B, &ep, &grp, &W};
    const int mb = ctx->score_min_blocks;
    if (g) {
        if (mb == 8) return launch_warps(ctx, score_kernel<true, 8>, B, wpb, smem, s, "score_grad", args);
        if (mb == 6) return launch_warps(ctx, score_kernel<true, 6>, B, wpb, smem, s, "score_grad", args);
        return launch_warps(ctx, score_kernel<true, 1>, B, wpb, smem, s, "score_grad", args);
    }
    if (mb == 8) return launch_warps(ctx, score_kernel<false, 8>, B, wpb, smem, s, "score", args);
    if (mb == 6) return launch_warps(ctx, score_kernel<false, 6>, B, wpb, smem, s, "score", args);
    return launch_warps(ctx, score_kernel<false, 1>, B, wpb, smem, s, "score", args);
}

cudaError_t launch_pose(dock_ctx *ctx, const LigandDev &L, const float *geno, int B, float *xyz, cudaStream_t s) {
    EvalLayout W = eval_layout(L.n_atoms, L.n_frag, L.nb8, false, 1);
    const int wpb = pick_warps(ctx, W);
    const size_t smem = (size_t)W.total * sizeof(float) * wpb;
    LigandDev l = L;
    const float *gp = geno;
    float *xp = xyz;
    void *args[] = {&l, &gp, &B, &xp, &W};
    return launch_warps(ctx, pose_kernel, B, wpb, smem, s, "pose", args);
}

int evaluator_smem_ok(dock_ctx *ctx, const EvalLayout &w, int warps) {
    return (size_t)w.total * sizeof(float) * warps <= ctx->smem_optin;
}

#include "rescore.cuh"

namespace {

__global__ void rescore64_kernel(LigandDev L, GridDev G, const float *__restrict__ geno, int B, double *E) {
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b < B) E[b] = rescore64_one(L, G, geno + (size_t)b * L.n_genes);
}

}  // namespace

cudaError_t launch_rescore64(dock_ctx *ctx, const LigandDev &L, const GridDev &G, const float *geno, int B, double *E,
                             cudaStream_t s) {
    if (B <= 0) return cudaSuccess;
    TimedLaunch tl;
    timing_begin(ctx, kernel_id(ctx, "rescore64"), s, &tl);
    rescore64_kernel<<<(B + 63) / 64, 64, 0, s>>>(L, G, geno, B, E);
    timing_end(ctx, s, &tl);
    ++ctx->launches;
    return cudaGetLastError();
}
