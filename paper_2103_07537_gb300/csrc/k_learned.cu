// Learned damping weights (beyond the paper: the paper fixes one damping of
// its block Gauss-Seidel smoother near 0.5 and shows that the value decides
// convergence for small viscosity, Sec. 5).  A network 8 -> 64 -> 64 -> 2
// (tanh) maps features of a level's matrix to the smoother damping of every
// node and field (head 0) and to the prolongator smoothing weight of every
// aggregate and field (head 1).
//   features       features_kernel, agg_features_kernel (FP64 math, FP32 out)
//   inference      mlp_forward_kernel: FP16 parameters, FP32 arithmetic
//   training       mlp_grad_kernel (+ deterministic reduction), adam_kernel
// The network is small (4882 parameters): the kernels stage the parameters
// in shared memory as FP32 and use plain FMA; rows are independent.
#include <cuda_fp16.h>

#include "common.cuh"

namespace bamg {

constexpr int kNF = BAMG_NFEAT, kNH = BAMG_MLP_H, kNO = BAMG_MLP_OUT;
constexpr int kOW1 = 0, kOB1 = kOW1 + kNH * kNF, kOW2 = kOB1 + kNH, kOB2 = kOW2 + kNH * kNH, kOW3 = kOB2 + kNH,
              kOB3 = kOW3 + kNO * kNH, kOXM = kOB3 + kNO, kOXS = kOXM + kNF;
static_assert(kOXS + kNF == BAMG_MLP_NPARAMS, "parameter layout");
static_assert(kOXM == BAMG_MLP_NTRAIN, "parameter layout");

// ---------------------------------------------------------------------------
// features of node i, field f (see amg_features in bamg.h); thread per node
// ---------------------------------------------------------------------------
template <int B, int FB>
__global__ void features_kernel(int n, const int* __restrict__ rp, const int* __restrict__ ci,
                                const double* __restrict__ vals, const int* __restrict__ agg,
                                const int* __restrict__ agg_cnt, int level, float* __restrict__ out, int* err) {
    constexpr int F = B / FB;
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    double d[F], o[F], c[F], tr[F];
#pragma unroll
    for (int f = 0; f < F; ++f) d[f] = o[f] = c[f] = tr[f] = 0.0;
    for (int k = rp[i]; k < rp[i + 1]; ++k) {
        const double* blk = vals + (size_t)k * B * B;
        const int j = ci[k];
#pragma unroll
        for (int f = 0; f < F; ++f) {
#pragma unroll
            for (int g = 0; g < F; ++g) {
                double s = 0.0;
                for (int r = 0; r < FB; ++r)
                    for (int cc = 0; cc < FB; ++cc) {
                        const double v = blk[(f * FB + r) * B + g * FB + cc];
                        s += v * v;
                    }
                const double nrm = sqrt(s);
                if (g != f) c[f] += nrm;
                else if (j == i) d[f] = nrm;
                else o[f] += nrm;
            }
            if (j == i)
                for (int r = 0; r < FB; ++r) tr[f] += blk[(f * FB + r) * B + f * FB + r];
        }
    }
    double mean_log = 0.0;
#pragma unroll
    for (int f = 0; f < F; ++f) {
        if (!(d[f] > 0.0)) {
            set_error(err, kDevSingularBlock);
            return;
        }
        mean_log += log(d[f]);
    }
    mean_log /= F;
    const int a = agg[i];
    const double lsz = log((double)agg_cnt[a]);
#pragma unroll
    for (int f = 0; f < F; ++f) {
        float* x = out + ((size_t)i * F + f) * kNF;
        const double ld = log(d[f]);
        x[0] = (float)ld;
        x[1] = (float)(o[f] / d[f]);
        x[2] = (float)(c[f] / (d[f] + o[f]));
        x[3] = (float)(ld - mean_log);
        x[4] = (float)(tr[f] / (sqrt((double)FB) * d[f]));
        x[5] = (float)lsz;
        x[6] = (float)level;
        x[7] = (float)f;
    }
}

__global__ void agg_count_kernel(int n, int nc, const int* __restrict__ agg, int* __restrict__ cnt, int* err) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int a = agg[i];
    if (a < 0 || a >= nc) {
        set_error(err, kDevBadPattern);
        return;
    }
    atomicAdd(cnt + a, 1);
}

// aggregate features: the mean of the member rows; thread per (I, f, m),
// members visited in ascending node order through the sorted member lists
__global__ void agg_features_kernel(int nc, int F, const int* __restrict__ agg_ptr, const int* __restrict__ members,
                                    const float* __restrict__ node_feat, float* __restrict__ out) {
    const long e = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= (long)nc * F * kNF) return;
    const int I = (int)(e / (F * kNF));
    const int w = (int)(e % (F * kNF));
    double s = 0.0;
    const int q0 = agg_ptr[I], q1 = agg_ptr[I + 1];
    for (int q = q0; q < q1; ++q) s += (double)node_feat[(size_t)members[q] * F * kNF + w];
    out[e] = (float)(s / (double)(q1 - q0));
}

int launch_features(int b, int fb, int n, const int* rp, const int* ci, const double* vals, const int* agg,
                    const int* agg_cnt, int level, float* out, int* err, cudaStream_t s) {
    if (n <= 0) return BAMG_OK;
    const int grid = ceil_div(n, 128);
    switch (b * 16 + fb) {
#define CASE(BB, FF)                                                                                     \
    case BB * 16 + FF:                                                                                   \
        features_kernel<BB, FF><<<grid, 128, 0, s>>>(n, rp, ci, vals, agg, agg_cnt, level, out, err);    \
        break;
        BAMG_BLOCK_SHAPES(CASE)
#undef CASE
        default: return BAMG_EUNSUPPORTED;
    }
    return launched(1);
}

int launch_agg_count(int n, int nc, const int* agg, int* cnt, int* err, cudaStream_t s) {
    BAMG_CUDA_TRY(cudaMemsetAsync(cnt, 0, sizeof(int) * (size_t)(nc > 0 ? nc : 1), s));
    if (n <= 0) return BAMG_OK;
    agg_count_kernel<<<ceil_div(n, 256), 256, 0, s>>>(n, nc, agg, cnt, err);
    return launched(1);
}

int launch_agg_features(int nc, int F, const int* agg_ptr, const int* members, const float* node_feat, float* out,
                        cudaStream_t s) {
    if (nc <= 0) return BAMG_OK;
    agg_features_kernel<<<ceil_div((long)nc * F * kNF, 256), 256, 0, s>>>(nc, F, agg_ptr, members, node_feat, out);
    return launched(1);
}

// ---------------------------------------------------------------------------
// network
// ---------------------------------------------------------------------------
__global__ void pack_half_kernel(const float* __restrict__ p, uint16_t* __restrict__ p16) {
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e < BAMG_MLP_NPARAMS) p16[e] = __half_as_ushort(__float2half_rn(p[e]));
}

__device__ __forceinline__ void stage_params(const uint16_t* __restrict__ p16, float* sp) {
    for (int e = threadIdx.x; e < BAMG_MLP_NPARAMS; e += blockDim.x) sp[e] = __half2float(__ushort_as_half(p16[e]));
    __syncthreads();
}

// forward pass of one training row: xh, and h1, h2 into shared-memory rows
__device__ __forceinline__ void row_forward(const float* __restrict__ sp, const float* __restrict__ x, float* xh,
                                            float* h1, float* h2, float* y) {
#pragma unroll
    for (int m = 0; m < kNF; ++m) xh[m] = (x[m] - sp[kOXM + m]) * sp[kOXS + m];
    for (int k = 0; k < kNH; ++k) {
        float a = 0.f;
#pragma unroll
        for (int m = 0; m < kNF; ++m) a = fmaf(sp[kOW1 + k * kNF + m], xh[m], a);
        h1[k] = tanhf(a + sp[kOB1 + k]);
    }
    float y0 = 0.f, y1 = 0.f;
    for (int j = 0; j < kNH; ++j) {
        float a = 0.f;
#pragma unroll
        for (int k = 0; k < kNH; ++k) a = fmaf(sp[kOW2 + j * kNH + k], h1[k], a);
        const float h = tanhf(a + sp[kOB2 + j]);
        h2[j] = h;
        y0 = fmaf(sp[kOW3 + j], h, y0);
        y1 = fmaf(sp[kOW3 + kNH + j], h, y1);
    }
    y[0] = y0 + sp[kOB3];
    y[1] = y1 + sp[kOB3 + 1];
}

// The same arithmetic as row_forward (every sum from 0 in ascending index
// order, bias added last) with the loops exchanged: h1[k] is produced one at
// a time and folded into the 64 accumulators of the second layer at once, so
// no activation array is indexed at run time and nothing spills.
__device__ __forceinline__ void row_infer(const float* __restrict__ sp, const float* __restrict__ x, float* y) {
    float xh[kNF], a2[kNH];
#pragma unroll
    for (int m = 0; m < kNF; ++m) xh[m] = (x[m] - sp[kOXM + m]) * sp[kOXS + m];
#pragma unroll
    for (int j = 0; j < kNH; ++j) a2[j] = 0.f;
    for (int k = 0; k < kNH; ++k) {
        float a = 0.f;
#pragma unroll
        for (int m = 0; m < kNF; ++m) a = fmaf(sp[kOW1 + k * kNF + m], xh[m], a);
        const float h = tanhf(a + sp[kOB1 + k]);
#pragma unroll
        for (int j = 0; j < kNH; ++j) a2[j] = fmaf(sp[kOW2 + j * kNH + k], h, a2[j]);
    }
    float y0 = 0.f, y1 = 0.f;
#pragma unroll
    for (int j = 0; j < kNH; ++j) {
        const float h = tanhf(a2[j] + sp[kOB2 + j]);
        y0 = fmaf(sp[kOW3 + j], h, y0);
        y1 = fmaf(sp[kOW3 + kNH + j], h, y1);
    }
    y[0] = y0 + sp[kOB3];
    y[1] = y1 + sp[kOB3 + 1];
}

// grid-stride over rows: each CTA stages the parameters once
__global__ void __launch_bounds__(128) mlp_forward_kernel(const uint16_t* __restrict__ p16, const float* __restrict__ x,
                                                          int n, float* __restrict__ y) {
    __shared__ float sp[BAMG_MLP_NPARAMS];
    stage_params(p16, sp);
    for (long r = (long)blockIdx.x * blockDim.x + threadIdx.x; r < n; r += (long)gridDim.x * blockDim.x) {
        float xr[kNF], out[kNO];
#pragma unroll
        for (int m = 0; m < kNF; ++m) xr[m] = x[r * kNF + m];
        row_infer(sp, xr, out);
        y[r * kNO] = out[0];
        y[r * kNO + 1] = out[1];
    }
}

int launch_mlp_forward(const uint16_t* p16, const float* x, int n, float* y, cudaStream_t s) {
    if (n <= 0) return BAMG_OK;
    const int grid = ceil_div(n, 128) < 152 * 4 ? ceil_div(n, 128) : 152 * 4;
    mlp_forward_kernel<<<grid, 128, 0, s>>>(p16, x, n, y);
    return launched(1);
}

int launch_pack_half(const float* p, uint16_t* p16, cudaStream_t s) {
    pack_half_kernel<<<ceil_div(BAMG_MLP_NPARAMS, 256), 256, 0, s>>>(p, p16);
    return launched(1);
}

// Gradient of the mean squared error over one tile of kTileRows rows.
// Phase 1, thread per row: forward, dL/dy, back through both tanh layers;
// the activations and pre-activation gradients of the tile go to shared
// memory.  Phase 2, all threads: the parameter gradients of the tile as
// sums over its rows in ascending order, written to partial[tile][NTRAIN].
constexpr int kTileRows = 64;
constexpr int kGradThreads = 256;
constexpr int kLd = kNH + 1;  // padded row stride of the activation tiles

struct GradSmem {
    float sp[BAMG_MLP_NPARAMS];
    float h1[kTileRows][kLd];
    float h2[kTileRows][kLd];
    float da1[kTileRows][kLd];
    float da2[kTileRows][kLd];
    float xh[kTileRows][kNF];
    float dy[kTileRows][kNO];
    float err2[kTileRows];
};

__global__ void __launch_bounds__(kGradThreads)
    mlp_grad_kernel(const uint16_t* __restrict__ p16, const float* __restrict__ x, const float* __restrict__ t,
                    const int* __restrict__ head, int n, float* __restrict__ partial, float* __restrict__ partial_loss) {
    extern __shared__ float4 smem_raw[];
    GradSmem& S = *reinterpret_cast<GradSmem*>(smem_raw);
    stage_params(p16, S.sp);
    const int tid = threadIdx.x;
    const long r0 = (long)blockIdx.x * kTileRows;
    if (tid < kTileRows) {
        const long r = r0 + tid;
        float xr[kNF], xh[kNF], y[kNO];
        float* h1 = S.h1[tid];
        float* h2 = S.h2[tid];
        const bool act = r < n;
#pragma unroll
        for (int m = 0; m < kNF; ++m) xr[m] = act ? x[r * kNF + m] : 0.f;
        row_forward(S.sp, xr, xh, h1, h2, y);
        float dy0 = 0.f, dy1 = 0.f, e2 = 0.f;
        if (act) {
            const int hd = head[r];
            const float e = (hd == 0 ? y[0] : y[1]) - t[r];
            e2 = e * e;
            const float g = 2.f * e / (float)n;
            dy0 = hd == 0 ? g : 0.f;
            dy1 = hd == 0 ? 0.f : g;
        }
        S.dy[tid][0] = dy0;
        S.dy[tid][1] = dy1;
        S.err2[tid] = e2;
#pragma unroll
        for (int m = 0; m < kNF; ++m) S.xh[tid][m] = xh[m];
        float* da2 = S.da2[tid];
        for (int j = 0; j < kNH; ++j) {
            const float g = dy0 * S.sp[kOW3 + j] + dy1 * S.sp[kOW3 + kNH + j];
            da2[j] = g * (1.f - h2[j] * h2[j]);
        }
        for (int k = 0; k < kNH; ++k) {
            float g = 0.f;
#pragma unroll 8
            for (int j = 0; j < kNH; ++j) g = fmaf(S.sp[kOW2 + j * kNH + k], da2[j], g);
            S.da1[tid][k] = g * (1.f - h1[k] * h1[k]);
        }
    }
    __syncthreads();
    float* out = partial + (size_t)blockIdx.x * BAMG_MLP_NTRAIN;
    // W2 and b2 (4096 + 64 outputs), W1 and b1 (512 + 64), W3 and b3 (128 + 2)
    for (int o = tid; o < BAMG_MLP_NTRAIN; o += kGradThreads) {
        float acc = 0.f;
        if (o >= kOW2 && o < kOB2) {
            const int j = (o - kOW2) / kNH, k = (o - kOW2) % kNH;
            for (int r = 0; r < kTileRows; ++r) acc = fmaf(S.da2[r][j], S.h1[r][k], acc);
        } else if (o >= kOB2 && o < kOW3) {
            const int j = o - kOB2;
            for (int r = 0; r < kTileRows; ++r) acc += S.da2[r][j];
        } else if (o < kOB1) {
            const int k = o / kNF, m = o % kNF;
            for (int r = 0; r < kTileRows; ++r) acc = fmaf(S.da1[r][k], S.xh[r][m], acc);
        } else if (o < kOW2) {
            const int k = o - kOB1;
            for (int r = 0; r < kTileRows; ++r) acc += S.da1[r][k];
        } else if (o < kOB3) {
            const int q = o - kOW3, oo = q / kNH, j = q % kNH;
            for (int r = 0; r < kTileRows; ++r) acc = fmaf(S.dy[r][oo], S.h2[r][j], acc);
        } else {
            const int oo = o - kOB3;
            for (int r = 0; r < kTileRows; ++r) acc += S.dy[r][oo];
        }
        out[o] = acc;
    }
    if (tid == 0) {
        float l = 0.f;
        for (int r = 0; r < kTileRows; ++r) l += S.err2[r];
        partial_loss[blockIdx.x] = l;
    }
}

// grad[o] = sum over tiles (ascending) of partial[tile][o]; loss likewise / n
__global__ void grad_reduce_kernel(int ntile, int n, const float* __restrict__ partial,
                                   const float* __restrict__ partial_loss, float* __restrict__ grad,
                                   float* __restrict__ loss) {
    const int o = blockIdx.x * blockDim.x + threadIdx.x;
    if (o < BAMG_MLP_NTRAIN) {
        float s = 0.f;
        for (int tt = 0; tt < ntile; ++tt) s += partial[(size_t)tt * BAMG_MLP_NTRAIN + o];
        grad[o] = s;
    }
    if (o == 0) {
        float s = 0.f;
        for (int tt = 0; tt < ntile; ++tt) s += partial_loss[tt];
        *loss = s / (float)n;
    }
}

size_t mlp_grad_workspace(int n) {
    const int ntile = ceil_div(n, kTileRows);
    return sizeof(float) * ((size_t)ntile * BAMG_MLP_NTRAIN + (size_t)ntile);
}

int launch_mlp_grad(const uint16_t* p16, const float* x, const float* t, const int* head, int n, float* grad,
                    float* loss, float* work, cudaStream_t s) {
    if (n < 1) return BAMG_EINVAL;
    const int ntile = ceil_div(n, kTileRows);
    const size_t smem = sizeof(GradSmem);
    // more than 48 KB of dynamic shared memory needs the opt-in (idempotent)
    BAMG_CUDA_TRY(cudaFuncSetAttribute(mlp_grad_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    float* partial = work;
    float* partial_loss = work + (size_t)ntile * BAMG_MLP_NTRAIN;
    mlp_grad_kernel<<<ntile, kGradThreads, smem, s>>>(p16, x, t, head, n, partial, partial_loss);
    grad_reduce_kernel<<<ceil_div(BAMG_MLP_NTRAIN, 256), 256, 0, s>>>(ntile, n, partial, partial_loss, grad, loss);
    return launched(2);
}

// Adam with bias-corrected moments on the trained parameters; c1 = 1 -
// beta1^t, c2 = 1 - beta2^t; then the FP16 copy of every parameter
__global__ void adam_kernel(float* __restrict__ p, uint16_t* __restrict__ p16, const float* __restrict__ g,
                            float* __restrict__ m, float* __restrict__ v, float lr, float beta1, float beta2,
                            float eps, float c1, float c2) {
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= BAMG_MLP_NPARAMS) return;
    if (e < BAMG_MLP_NTRAIN) {
        const float gg = g[e];
        const float mm = beta1 * m[e] + (1.f - beta1) * gg;
        const float vv = beta2 * v[e] + (1.f - beta2) * gg * gg;
        m[e] = mm;
        v[e] = vv;
        p[e] -= lr * (mm / c1) / (sqrtf(vv / c2) + eps);
    }
    p16[e] = __half_as_ushort(__float2half_rn(p[e]));
}

int launch_adam(float* p, uint16_t* p16, const float* g, float* m, float* v, float lr, float beta1, float beta2,
                float eps, float c1, float c2, cudaStream_t s) {
    adam_kernel<<<ceil_div(BAMG_MLP_NPARAMS, 256), 256, 0, s>>>(p, p16, g, m, v, lr, beta1, beta2, eps, c1, c2);
    return launched(1);
}

// ---------------------------------------------------------------------------
// weights of a level from the network outputs (same ranges as mlp_clip):
// out64[r] = clip_head(y[r][head]); *any = 1 if some value is nonzero
// ---------------------------------------------------------------------------
__device__ __forceinline__ double clip_weight(int head, double w) {
    if (head == 0) return !(w >= 0.05) ? 0.05 : (w > 1.5 ? 1.5 : w);
    return !(w >= 0.05) ? 0.0 : (w > 1.5 ? 1.5 : w);
}

__global__ void omega_from_mlp_kernel(int rows, int head, const float* __restrict__ y, double* __restrict__ out,
                                      int* __restrict__ any) {
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= rows) return;
    const double w = clip_weight(head, (double)y[(size_t)r * kNO + head]);
    out[r] = w;
    if (any && w > 0.0) atomicOr(any, 1);
}

int launch_omega_from_mlp(int rows, int head, const float* y, double* out, int* any, cudaStream_t s) {
    if (rows <= 0) return BAMG_OK;
    omega_from_mlp_kernel<<<ceil_div(rows, 256), 256, 0, s>>>(rows, head, y, out, any);
    return launched(1);
}

__global__ void fill_kernel(long m, double v, double* __restrict__ out) {
    const long e = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (e < m) out[e] = v;
}

int launch_fill(long m, double v, double* out, cudaStream_t s) {
    if (m <= 0) return BAMG_OK;
    fill_kernel<<<ceil_div(m, 256), 256, 0, s>>>(m, v, out);
    return launched(1);
}

}  // namespace bamg

extern "C" double mlp_clip(int head, double w) {
    if (head == 0) return !(w >= 0.05) ? 0.05 : (w > 1.5 ? 1.5 : w);
    return !(w >= 0.05) ? 0.0 : (w > 1.5 ? 1.5 : w);
}
