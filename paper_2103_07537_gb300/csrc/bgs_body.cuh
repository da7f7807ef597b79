// Device-side building blocks of the block Gauss-Seidel smoother of
// Algorithm 1 (Sec. 4.3.2) shared by the per-colour kernels (k_solve.cu) and
// the persistent sweep kernel (k_sweep.cu): vector loads with an optional
// L2-coherent path and the per-block accumulation of one field step.
#pragma once

#include "common.cuh"

namespace bamg {

// ---------------------------------------------------------------------------
// loads of B consecutive values of a vector (coherent variant for the tail)
// ---------------------------------------------------------------------------
template <typename T, int B, bool CG>
__device__ __forceinline__ void load_vec(const T* __restrict__ p, T (&out)[B]) {
    if constexpr (!CG) {
        load_row<T, B>(p, out);
    } else {
        constexpr int bytes_row = B * (int)sizeof(T);
        if constexpr (sizeof(T) == 4 && bytes_row % 16 == 0) {
#pragma unroll
            for (int c = 0; c < B; c += 4) {
                float4 v = __ldcg(reinterpret_cast<const float4*>(p + c));
                out[c] = v.x;
                out[c + 1] = v.y;
                out[c + 2] = v.z;
                out[c + 3] = v.w;
            }
        } else if constexpr (bytes_row % 16 == 0 || (sizeof(T) == 4 && bytes_row % 8 == 0)) {
            using V2 = typename VecOf<T>::v2;
#pragma unroll
            for (int c = 0; c < B; c += 2) {
                V2 v = __ldcg(reinterpret_cast<const V2*>(p + c));
                out[c] = v.x;
                out[c + 1] = v.y;
            }
        } else {
#pragma unroll
            for (int c = 0; c < B; ++c) out[c] = __ldcg(p + c);
        }
    }
}

template <typename T, bool CG>
__device__ __forceinline__ T ld1(const T* p) {
    if constexpr (CG) return __ldcg(p);
    else return *p;
}

// one block of a field step of the smoother: acc += A_{f,*}[i,j] x_in,j (x_in
// plus P uc when fused), and acc += A_ff[i,j] x~_j when j precedes i in the
// colour order (x~ of later colours is stale and masked); arow = row f0 + r of
// the block.  Forced inline so that arow stays in registers.
// (CG: x~ read through L2 (it is written in the same launch); CGX: the same
// for x_in and uc, which only the tail kernel writes in the same launch)
template <typename T, int B, int FB, bool CG, bool CGX = CG>
__device__ __forceinline__ void bgs_block(const BgsArgs& a, const T* xt, const T* x_in, const T* uc, int j,
                                          const T (&arow)[B], bool lower, int ag, T& acc) {
    T tv[FB];
    if (lower) load_vec<T, FB, CG>(xt + (size_t)j * FB, tv);
    if (x_in) {
        T xv[B];
        load_vec<T, B, CGX>(x_in + (size_t)j * B, xv);
        if (uc) {
            T pv[B];
            load_vec<T, B, CGX>(uc + (size_t)ag * B, pv);
#pragma unroll
            for (int c = 0; c < B; ++c) xv[c] += pv[c];
        }
#pragma unroll
        for (int c = 0; c < B; ++c) acc = fma(arow[c], xv[c], acc);
    }
    if (lower) {
        // the field-f columns of the row, picked by selects over compile-time
        // register indices (an index computed from the field would put arow
        // in local memory)
#pragma unroll
        for (int c = 0; c < FB; ++c) {
            T av = arow[c];
#pragma unroll
            for (int ff = 1; ff < B / FB; ++ff) av = (ff == a.field) ? arow[ff * FB + c] : av;
            acc = fma(av, tv[c], acc);
        }
    }
}

}  // namespace bamg
