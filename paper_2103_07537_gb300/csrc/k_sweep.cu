// Persistent multicolour sweep: every colour of one field step of the block
// Gauss-Seidel smoother (Algorithm 1, Sec. 4.3.2) in one launch.
//
// A field step visits the colours in order; node i of colour c needs x~ of
// its neighbours of lower colour (the blocks flagged in lowk) and nothing of
// later colours.  Launched per colour, each launch covers a fraction of the
// level (1/8 of the 3D rows) and pays its own ramp-up and drain.  Here the
// nodes of every colour are cut into tiles (runs of NTILE consecutive
// entries of the colour-ordered node list), numbered colour by colour, and
// the CTAs of one resident grid take tiles in that order from an atomic
// ticket.  Before a tile is computed its CTA waits until every tile holding
// one of its lower-colour neighbours is done (per-tile flags; the tile ranges
// per lower colour are found once at setup).  A tile only waits for tiles
// with smaller numbers, and those were taken earlier by CTAs that are
// running, so the wait always ends without any residency guarantee; every
// wait is bounded all the same (kSweepSpins polls, then kDevTimeout).
//
// Flags carry the launch's epoch (ctrl[2] + 1): the CTA that leaves last
// resets the ticket and the exit count and moves the epoch, so the flags and
// the control words need no clearing between launches or graph replays.  x~
// written in the launch is read through L2 (ld.global.cg); the producer
// orders its writes before the flag by a barrier and a fence (as a grid
// barrier does), the consumer's polling warp by a fence after the flags, and
// the CTA by a barrier.
// The arithmetic per node is that of the thread-per-row kernel of k_solve.cu
// (same sums in the same order), so the sweep gives the same values.
#include "bgs_body.cuh"
#include "common.cuh"

namespace bamg {

constexpr long kSweepSpins = 1L << 22;  // polls of one flag (a 64 ns sleep and an L2 round trip each): seconds

__device__ __forceinline__ unsigned ld_acquire_u32(const unsigned* p) {
    unsigned v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ void st_release_u32(unsigned* p, unsigned v) {
    asm volatile("st.release.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

// threads per CTA and nodes per tile for fb x fb sub-blocks (the CTA covers a
// tile in NTILE / (threads / (FB * G)) passes)
template <int FB>
struct SweepShape {
    static constexpr int kThreads = RowThreads<FB>::kThreads;
    // at least 64 nodes, a whole number of passes of one thread per row
    static constexpr int kTile = (kThreads / FB) * ((64 + kThreads / FB - 1) / (kThreads / FB));
};

int sweep_tile_nodes(int fb) {
    switch (fb) {
        case 1: return SweepShape<1>::kTile;
        case 2: return SweepShape<2>::kTile;
        case 3: return SweepShape<3>::kTile;
        case 4: return SweepShape<4>::kTile;
        case 5: return SweepShape<5>::kTile;
        case 6: return SweepShape<6>::kTile;
        case 7: return SweepShape<7>::kTile;
        case 8: return SweepShape<8>::kTile;
        default: return 0;
    }
}

template <typename T, int B, int FB, int G, bool FM>
__global__ void __launch_bounds__(SweepShape<FB>::kThreads) bgs_sweep_kernel(BgsArgs a, SweepArgs sw) {
    constexpr int NT = SweepShape<FB>::kThreads;
    constexpr int PER_PASS = NT / (FB * G);
    constexpr int NTILE = SweepShape<FB>::kTile;
    constexpr int PASSES = NTILE / PER_PASS;
    static_assert(NT % (FB * G) == 0 && NTILE % PER_PASS == 0, "tile shape");
    __shared__ T sh_t[PER_PASS * FB];
    __shared__ int s_cptr[kSweepMaxColours + 1], s_tptr[kSweepMaxColours + 1];
    __shared__ int s_lo[kSweepMaxColours], s_hi[kSweepMaxColours];
    __shared__ int s_tile;
    __shared__ unsigned s_want;
    const int tid = threadIdx.x;
    const int nloc = tid / (FB * G);
    const int w = tid - nloc * (FB * G);
    const int r = w / G, sl = w - r * G;  // scalar row of the node, slice of the row's blocks
    const int nc = sw.c_hi - sw.c_lo;
    const int f0 = a.field * FB;
    const T* __restrict__ vals = static_cast<const T*>(a.vals);
    const T* __restrict__ x_in = static_cast<const T*>(a.x_in);
    const T* __restrict__ uc = static_cast<const T*>(a.uc);
    const T* xt = static_cast<const T*>(a.xt);  // written in this launch: read through L2
    // colour and tile ranges of the step (fixed for the level)
    for (int q = tid; q <= nc; q += NT) {
        s_cptr[q] = __ldg(sw.colour_ptr + sw.c_lo + q);
        s_tptr[q] = __ldg(sw.tile_ptr + sw.c_lo + q);
    }
    pdl_wait();  // the previous kernel (possibly a sweep on these control words) has finished
    pdl_trigger();
    if (tid == 0) s_want = ld_acquire_u32(sw.ctrl + 2) + 1u;
    __syncthreads();
    const unsigned want = s_want;
    const int t_first = s_tptr[0], t_end = s_tptr[nc];
    for (;;) {
        if (tid == 0) s_tile = t_first + (int)atomicAdd(sw.ctrl, 1u);
        __syncthreads();
        const int tile = s_tile;
        if (tile >= t_end) break;  // uniform over the CTA
        int cl = 0;  // colour of the tile, relative to c_lo
        while (cl + 1 < nc && s_tptr[cl + 1] <= tile) ++cl;
        if (tid < cl) {
            s_lo[tid] = __ldg(sw.dep_lo + (size_t)tile * sw.C + sw.c_lo + tid);
            s_hi[tid] = __ldg(sw.dep_hi + (size_t)tile * sw.C + sw.c_lo + tid);
        }
        __syncthreads();
        // wait for the tiles of the lower-colour neighbours: the first warp
        // polls (relaxed loads, each lane a share of the flags, a short sleep
        // between polls so that the waiting CTAs do not flood L2), then one
        // fence orders the flags before the CTA's reads; a timeout anywhere
        // ends every wait
        if (tid < 32) {
            for (int cc = 0; cc < cl; ++cc) {
                const int lo = s_lo[cc], hi = s_hi[cc];
                for (int q = lo + tid; q <= hi; q += 32) {
                    long spins = 0;
                    while (*reinterpret_cast<volatile const unsigned*>(sw.flags + q) != want) {
                        if (++spins > kSweepSpins) {
                            set_error(sw.err, kDevTimeout);
                            break;
                        }
                        if ((spins & 255) == 0 && *reinterpret_cast<volatile int*>(sw.err) != 0) break;
                        __nanosleep(64);
                    }
                }
            }
            __threadfence();
        }
        __syncthreads();
        const int pos0 = s_cptr[cl] + (tile - s_tptr[cl]) * NTILE;
        const int pend = s_cptr[cl + 1];
#pragma unroll 1
        for (int pass = 0; pass < PASSES; ++pass) {
            const int p = pos0 + pass * PER_PASS + nloc;
            const bool act = p < pend;
            int i = 0;
            T acc = T(0);
            if (act) {
                i = __ldg(a.nodes + p);
                const int k0 = __ldg(a.rp + i), k1 = __ldg(a.rp + i + 1);
                const T* vb = vrow<T, B, FB, FM>(vals, k0, k1, k0, f0 + r);
                constexpr int VS = vstride<T, B, FB, FM>();
#pragma unroll(G > 1 ? 8 : 4)
                for (int k = k0 + sl; k < k1; k += G) {
                    const bool lower = __ldg(a.lowk + k) != 0;
                    if (!x_in && !lower) continue;
                    const int j = __ldg(a.ci + k);
                    T arow[B];
                    load_row<T, B>(vb + (size_t)(k - k0) * VS, arow);
                    bgs_block<T, B, FB, true, false>(a, xt, x_in, uc, j, arow, lower,
                                                     (x_in && uc) ? __ldg(a.agg + j) : 0, acc);
                }
            }
            if constexpr (G > 1) {  // the G slices of a row are consecutive lanes of one warp
#pragma unroll
                for (int o = G / 2; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
            }
            if (sl == 0) sh_t[nloc * FB + r] = (act ? static_cast<const T*>(a.rhs)[(size_t)i * B + f0 + r] - acc : T(0));
            __syncthreads();
            if (act && sl == 0) {
                const T* D = static_cast<const T*>(a.dinv) + ((size_t)i * a.F + a.field) * FB * FB + (size_t)r * FB;
                T xn = T(0);
#pragma unroll
                for (int c = 0; c < FB; ++c) xn = fma(__ldg(D + c), sh_t[nloc * FB + c], xn);
                static_cast<T*>(a.xt)[(size_t)i * FB + r] = xn;
                T* __restrict__ x_out = static_cast<T*>(a.x_out);
                const T om =
                    a.omega_node ? static_cast<const T*>(a.omega_node)[(size_t)i * a.F + a.field] : T(a.omega);
                const int ag = (x_in && uc) ? __ldg(a.agg + i) : 0;
                for (int m = 0; m < a.F; ++m) {
                    const size_t e = (size_t)i * B + m * FB + r;
                    T v = x_in ? x_in[e] : T(0);
                    if (x_in && uc) v += uc[(size_t)ag * B + m * FB + r];
                    if (m == a.field) v = fma(om, xn, v);
                    x_out[e] = v;
                }
            }
            __syncthreads();  // sh_t is reused by the next pass
        }
        // publish the tile: every thread's writes, then the flag
        if (tid == 0) {
            __threadfence();
            st_release_u32(sw.flags + tile, want);
        }
    }
    // the last CTA to leave resets the ticket and the exit count, then moves
    // the epoch (no CTA of this launch takes a ticket after its exit)
    if (tid == 0) {
        __threadfence();
        if (atomicAdd(sw.ctrl + 1, 1u) == gridDim.x - 1) {
            sw.ctrl[0] = 0u;
            sw.ctrl[1] = 0u;
            __threadfence();
            atomicAdd(sw.ctrl + 2, 1u);
        }
    }
}

// resident CTAs of one kernel instance on the whole device (computed once)
template <class K>
static int resident_ctas(K kernel, int threads) {
    int dev = 0, sms = 0, per_sm = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) !=
                                                     cudaSuccess ||
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, threads, 0) != cudaSuccess)
        return 0;
    return sms * per_sm;
}

template <typename T, int B, int FB, int G, bool FM>
static int launch_sweep_instance(const BgsArgs& a, const SweepArgs& sw, int tiles, cudaStream_t s) {
    static const int resident = resident_ctas(bgs_sweep_kernel<T, B, FB, G, FM>, SweepShape<FB>::kThreads);
    if (resident <= 0) return BAMG_ECUDA;
    const int grid = tiles < resident ? tiles : resident;
    if (launch_k(bgs_sweep_kernel<T, B, FB, G, FM>, grid, SweepShape<FB>::kThreads, 0, s, a, sw) != cudaSuccess)
        return BAMG_ECUDA;
    return launched(1);
}

template <typename T>
int launch_bgs_sweep(int b, int fb, const BgsArgs& a, const SweepArgs& sw, int tiles, int g4, cudaStream_t s) {
    if (tiles <= 0) return BAMG_OK;
    if (sw.c_hi - sw.c_lo > kSweepMaxColours) return BAMG_EUNSUPPORTED;
    switch (b * 16 + fb) {
#define CASE(BB, FF)                                                                                           \
    case BB * 16 + FF: {                                                                                       \
        constexpr bool kFm = HasFm<T, BB, FF>::value;                                                         \
        if (g4)                                                                                                \
            return (a.fm && kFm) ? launch_sweep_instance<T, BB, FF, 4, kFm>(a, sw, tiles, s)                  \
                                 : launch_sweep_instance<T, BB, FF, 4, false>(a, sw, tiles, s);               \
        return (a.fm && kFm) ? launch_sweep_instance<T, BB, FF, 1, kFm>(a, sw, tiles, s)                      \
                             : launch_sweep_instance<T, BB, FF, 1, false>(a, sw, tiles, s);                   \
    }
        BAMG_BLOCK_SHAPES(CASE)
#undef CASE
        default: return BAMG_EUNSUPPORTED;
    }
}
template int launch_bgs_sweep<double>(int, int, const BgsArgs&, const SweepArgs&, int, int, cudaStream_t);
template int launch_bgs_sweep<float>(int, int, const BgsArgs&, const SweepArgs&, int, int, cudaStream_t);

// ---------------------------------------------------------------------------
// setup: the tiles of a level and their dependencies
// ---------------------------------------------------------------------------
// tile of every node: position p of colour c lies in tile
// tile_ptr[c] + (p - colour_ptr[c]) / ntile
__global__ void sweep_tile_of_kernel(int n, const int* __restrict__ nodes, const int* __restrict__ colour,
                                     const int* __restrict__ colour_ptr, const int* __restrict__ tile_ptr, int ntile,
                                     int* __restrict__ tile_of) {
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= n) return;
    const int i = nodes[p];
    const int c = colour[i];
    tile_of[i] = tile_ptr[c] + (p - colour_ptr[c]) / ntile;
}

// dep_lo / dep_hi [tile][colour]: the smallest and largest tile of that
// colour holding a neighbour whose x~ a node of the tile reads (lowk)
__global__ void sweep_deps_kernel(int n, const int* __restrict__ rp, const int* __restrict__ ci,
                                  const unsigned char* __restrict__ lowk, const int* __restrict__ colour,
                                  const int* __restrict__ tile_of, int C, int* __restrict__ dep_lo,
                                  int* __restrict__ dep_hi) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const size_t ti = (size_t)tile_of[i] * C;
    for (int k = rp[i]; k < rp[i + 1]; ++k) {
        if (!lowk[k]) continue;
        const int j = ci[k];
        const int tj = tile_of[j];
        atomicMin(dep_lo + ti + colour[j], tj);
        atomicMax(dep_hi + ti + colour[j], tj);
    }
}

int sweep_plan(int n, int C, int ntile, const int* nodes, const int* colour, const int* colour_ptr,
               const int* tile_ptr, const int* rp, const int* ci, const unsigned char* lowk, int n_tiles,
               int* tile_of, int* dep_lo, int* dep_hi, cudaStream_t s) {
    if (n <= 0) return BAMG_OK;
    BAMG_CUDA_TRY(cudaMemsetAsync(dep_lo, 0x7f, sizeof(int) * (size_t)n_tiles * C, s));
    BAMG_CUDA_TRY(cudaMemsetAsync(dep_hi, 0xff, sizeof(int) * (size_t)n_tiles * C, s));
    sweep_tile_of_kernel<<<ceil_div(n, 256), 256, 0, s>>>(n, nodes, colour, colour_ptr, tile_ptr, ntile, tile_of);
    sweep_deps_kernel<<<ceil_div(n, 256), 256, 0, s>>>(n, rp, ci, lowk, colour, tile_of, C, dep_lo, dep_hi);
    return launched(2);
}

}  // namespace bamg
