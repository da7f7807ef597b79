// Shared device helpers and internal declarations of the bamg CUDA library.
// Target: sm_103a (GB300).  No code here is shared with the CPU oracle.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <vector>

#include "bamg.h"

namespace bamg {

constexpr int kWarp = 32;

// Every (b, fb) block shape the cycle's kernels are instantiated for: b dofs
// per node in b / fb field blocks of fb dofs (amg_setup accepts exactly these)
#define BAMG_BLOCK_SHAPES(M) \
    M(1, 1) M(2, 2) M(3, 3) M(4, 4) M(5, 5) M(6, 6) M(7, 7) M(8, 8) M(4, 2) M(6, 3) M(6, 2) M(8, 4) M(8, 2)

// threads per CTA of the kernels with FB (or FB x 4) threads per node: a
// multiple of FB * 4 and of the warp, so that no node is split between CTAs
template <int FB>
struct RowThreads {
    static constexpr int kThreads = (FB == 3 || FB == 6) ? 192 : FB == 5 ? 160 : FB == 7 ? 224 : 256;
    static_assert(kThreads % (FB * 4) == 0 && kThreads % 32 == 0, "threads per CTA");
};
constexpr int kMaxLevels = 16;
constexpr int kMaxRestart = 64;
constexpr int kMaxB = 8;

// device error flag values (first error wins, atomicCAS from 0)
enum DevErr : int {
    kDevOk = 0,
    kDevSingularBlock = 1,
    kDevSingularCoarse = 2,
    kDevBadPattern = 3,   // unsorted columns / missing diagonal / out-of-range index
    kDevRowTooLong = 4,   // a coarse row exceeded the RAP row capacity
    kDevNonFinite = 5,
    kDevTimeout = 6,      // a bounded wait of a cooperative kernel ran out
};

__device__ __forceinline__ void set_error(int* flag, int code) { atomicCAS(flag, 0, code); }

// Barrier over every CTA of a cooperative launch: an arrival counter and a
// generation word in global memory (bar[0], bar[1], zero before the first
// launch; the last arriver resets the counter before it moves the
// generation, so the pair is ready for the next barrier and launch).  Thread
// 0 of each CTA spins on the generation; a wait beyond kBarrierSpins sets
// kDevTimeout and returns false, and the caller's CTA leaves, so the others
// run out at their next barrier and the kernel always ends.
constexpr long kBarrierSpins = 1L << 24;  // one L2 round trip per spin: well over a second

// Scalar row rr of block k of block row [k0, k1) in a level's values.  FP64
// values (the setup's and the outer SpMV's) are block-major: block k holds
// its B x B entries row by row.  The FP32 copy of a level larger than L2 in a
// cycle with F > 1 fields is field-major (fm) inside each block row: the FB
// rows of field f of all the row's blocks are contiguous (field 0 of every
// block, then field 1, ...), so a field step of the smoother streams one
// contiguous run per node instead of every other FB x B piece of the blocks.
// (On L2-resident levels the block-major copy measured faster.)
// (FM: the kernel instance for field-major values; launchers pick it from the
// level's flag, so block-major code is compiled exactly as without it)
template <typename T, int B, int FB>
struct HasFm {
    static constexpr bool value = sizeof(T) == 4 && FB < B;
};
template <typename T, int B, int FB, bool FM>
__host__ __device__ constexpr int vstride() {
    return (FM && HasFm<T, B, FB>::value) ? FB * B : B * B;  // same row of consecutive blocks
}
template <typename T, int B, int FB, bool FM>
__host__ __device__ __forceinline__ const T* vrow(const T* vals, int k0, int k1, int k, int rr) {
    if constexpr (FM && HasFm<T, B, FB>::value) {
        const int f = rr / FB, r = rr - f * FB;
        return vals + (size_t)k0 * B * B + ((size_t)f * (k1 - k0) + (k - k0)) * (FB * B) + (size_t)r * B;
    } else {
        return vals + (size_t)k * B * B + (size_t)rr * B;
    }
}

// Block-wide sums of the first gn of G values per thread (NT threads): the
// values go to shared memory (one row of G + 1 per thread), thread t adds
// value t % G over the G rows of slice t / G (S = NT / G slices) in row
// order, and thread g < gn adds the S slice sums in slice order and returns
// the total (a fixed order).  About G + S adds per thread, where a shuffle
// tree per value issues 5 adds per value in every thread: on GB300 (2 FP64
// operations per clock per SM) that work rivals the dot products themselves.
// sh: NT * (G + 1) + S * (G + 1) doubles.
template <int G, int NT>
__device__ __forceinline__ double block_sums(const double (&v)[G], int gn, double* sh) {
    constexpr int S = NT / G;
    static_assert(NT % G == 0, "NT must be a multiple of G");
    const int t = threadIdx.x;
    double* rows = sh;                      // [NT][G + 1]
    double* part = sh + NT * (G + 1);       // [S][G + 1]
#pragma unroll
    for (int g = 0; g < G; ++g)
        if (g < gn) rows[t * (G + 1) + g] = v[g];
    __syncthreads();
    {
        const int g = t % G, sl = t / G;
        if (g < gn) {
            double s = 0.0;
#pragma unroll 4
            for (int i = 0; i < G; ++i) s += rows[(sl * G + i) * (G + 1) + g];
            part[sl * (G + 1) + g] = s;
        }
    }
    __syncthreads();
    double tot = 0.0;
    if (t < gn)
        for (int sl = 0; sl < S; ++sl) tot += part[sl * (G + 1) + t];
    __syncthreads();  // sh is reused by the next call
    return tot;
}

__device__ __forceinline__ bool grid_barrier(unsigned* bar, int* err) {
    __shared__ int s_ok;
    __syncthreads();
    if (threadIdx.x == 0) {
        s_ok = 1;
        volatile unsigned* gen = bar + 1;
        const unsigned g = *gen;
        __threadfence();
        if (atomicAdd(bar, 1u) + 1u == gridDim.x) {
            bar[0] = 0u;  // nobody arrives again before the generation moves
            __threadfence();
            atomicAdd(bar + 1, 1u);
        } else {
            long spins = 0;
            while (*gen == g) {
                if (++spins > kBarrierSpins) {
                    set_error(err, kDevTimeout);
                    s_ok = 0;
                    break;
                }
            }
        }
        __threadfence();
    }
    __syncthreads();
    return s_ok != 0;
}

template <typename T>
struct VecOf;
template <>
struct VecOf<double> {
    using v2 = double2;
};
template <>
struct VecOf<float> {
    using v2 = float2;
};

// Load the B contiguous values starting at p (p aligned to the block-row
// start; rows of B values start at multiples of B elements inside blocks of
// B*B elements, blocks start at multiples of B*B elements, base 256-aligned).
// Uses the widest vector load that keeps every row start aligned.
template <typename T, int B>
__device__ __forceinline__ void load_row(const T* __restrict__ p, T (&out)[B]) {
    constexpr int bytes_row = B * (int)sizeof(T);
    if constexpr (sizeof(T) == 4 && bytes_row % 16 == 0) {
#pragma unroll
        for (int c = 0; c < B; c += 4) {
            float4 v = *reinterpret_cast<const float4*>(p + c);
            out[c] = v.x;
            out[c + 1] = v.y;
            out[c + 2] = v.z;
            out[c + 3] = v.w;
        }
    } else if constexpr (bytes_row % 16 == 0 || (sizeof(T) == 4 && bytes_row % 8 == 0)) {
        using V2 = typename VecOf<T>::v2;
#pragma unroll
        for (int c = 0; c < B; c += 2) {
            V2 v = *reinterpret_cast<const V2*>(p + c);
            out[c] = v.x;
            out[c + 1] = v.y;
        }
    } else {
#pragma unroll
        for (int c = 0; c < B; ++c) out[c] = p[c];
    }
}

template <typename T>
__device__ __forceinline__ T warp_sum(T v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

inline int ceil_div(long a, long b) { return (int)((a + b - 1) / b); }

// Programmatic dependent launch (sm_90 and later).  A V-cycle kernel launched
// with the programmatic-serialization attribute may be scheduled while its
// predecessor in the stream drains; before reading anything an earlier kernel
// wrote it must pass pdl_wait(), which returns once the predecessor grid has
// completed and its writes are visible (a hardware dependency, no polling).
// pdl_trigger() lets the successor be scheduled early; it is issued right
// after pdl_wait(), so at most one kernel ahead is resident and waiting (a
// trigger at kernel entry let a chain of future kernels occupy the SMs and
// measured slower).  Without the attribute both are no-ops.  Data that is
// constant during a cycle (matrices, inverses, colour lists, dampings) may be
// read before pdl_wait().
__device__ __forceinline__ void pdl_trigger() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }

// launch mode of the V-cycle kernels on this host thread: set by the library
// around the launches (or the graph capture) of one cycle
extern thread_local bool t_pdl;

// kernel launch with the programmatic-serialization attribute when t_pdl is set
template <typename... KArgs, typename... Args>
inline cudaError_t launch_k(void (*kernel)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t s,
                            Args... args) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = t_pdl ? 1 : 0;
    return cudaLaunchKernelEx(&cfg, kernel, static_cast<KArgs>(args)...);
}

// counts kernel launches (defined in capi.cu); while a CUDA graph is being
// captured on this thread the count goes to the graph instead
void note_launch(int count = 1);
// status after k kernel launches (counted)
inline int launched(int k) {
    note_launch(k);
    return cudaGetLastError() == cudaSuccess ? BAMG_OK : BAMG_ECUDA;
}

}  // namespace bamg

// ---------------------------------------------------------------------------
// internal launchers (host functions, defined in the k_*.cu files)
// ---------------------------------------------------------------------------
namespace bamg {

// ---- solve-phase kernels (k_solve.cu) ----
// y = A x (+ optional: y = rhs - A x when rhs != nullptr).  T = matrix/vector
// type; vals in the layout of vrow for (b, fb) (fb = b: block-major)
template <typename T>
int launch_spmv(int b, int fb, int fm, int n, const int* rp, const int* ci, const T* vals, const T* x, const T* rhs,
                T* y, cudaStream_t s);
// rc[I*b+d] = sum over members m of aggregate I (ascending) of res[m*b+d]
template <typename T>
int launch_restrict(int b, int nc, const int* agg_ptr, const int* members, const T* res, T* rc,
                    cudaStream_t s);
// u[i*b+d] += uc[agg[i]*b+d]
template <typename T>
int launch_prolong(int b, int n, const int* agg, const T* uc, T* u, cudaStream_t s);
// y[i*b+d] = x[i*b+d] (+ uc[agg[i]*b+d] when uc is set), or 0 without x
template <typename T>
int launch_copy_prolong(int b, int n, const int* agg, const T* x, const T* uc, T* y, cudaStream_t s);
// One colour of one field step of the block Gauss-Seidel smoother.
struct BgsArgs {
    int n_in_colour = 0;
    const int* nodes = nullptr;    // node ids of this colour
    int colour = 0;                // colour index (neighbours of lower colour carry x~)
    const int* colours = nullptr;  // colour of every node
    const int* rp = nullptr;
    const int* ci = nullptr;
    const void* vals = nullptr;
    const void* dinv = nullptr;    // [n][F][fb*fb]
    const void* rhs = nullptr;
    const void* x_in = nullptr;    // nullptr = zero vector
    void* x_out = nullptr;
    void* xt = nullptr;            // [n][fb]
    const void* uc = nullptr;      // optional: coarse correction added to x_in on the fly (x_in + P uc)
    const int* agg = nullptr;      // aggregate of every node (with uc)
    int field = 0;
    int F = 1;
    double omega = 0.5;
    const void* omega_node = nullptr;  // optional: damping of every node and field ([n][F], type T) in place of omega
    // 1 where block k of row i has a column j != i of lower colour than i
    // (fixed for the level: no gather of the neighbour's colour in the cycle)
    const unsigned char* lowk = nullptr;
    int fm = 0;  // vals in the field-major layout (see vrow)
};
template <typename T>
int launch_bgs_colour(int b, int fb, const BgsArgs& a, cudaStream_t s);
// the same step with four warps per node, one node per CTA (long rows, small colours)
template <typename T>
int launch_bgs_colour_wide(int b, int fb, const BgsArgs& a, cudaStream_t s);
// FP32 copy of block-major FP64 values in the field-major layout of vrow
int launch_convert_fieldmajor(int n, int b, int fb, const int* rp, const double* x, float* y, cudaStream_t s);
// lowk[k] = 1 where block k of row i has a column j != i with colour[j] < colour[i]
int launch_lower_flags(int n, const int* rp, const int* ci, const int* colour, unsigned char* lowk, cudaStream_t s);
// thread-per-row variants (more loads in flight per warp; for large levels)
template <typename T>
// variant 0: one thread per scalar row; 1: as 0 in CTAs of half the threads (a
// small colour spread over more SMs); 2: four lanes per scalar row, each
// taking every fourth block (shorter dependent-load chains per thread)
int launch_bgs_colour_tpr(int b, int fb, const BgsArgs& a, cudaStream_t s, int variant = 0);
// G = 8 or 16 lanes per node, each taking whole blocks (block-split; shapes
// with fb * b <= 16, else BAMG_EUNSUPPORTED)
bool bsp_supported(int b, int fb);
template <typename T>
int launch_bgs_colour_bsp(int b, int fb, const BgsArgs& a, int G, cudaStream_t s);
// fields of unequal size run padded (k_pad.cu): padded dof q of a node is
// place q % fmax of field q / fmax; dummy places have src -1
struct PadMap {
    int b = 0, bp = 0;            // dofs per node: given, padded
    signed char src[kMaxB] = {};  // padded dof -> given dof (-1: dummy)
    signed char dst[kMaxB] = {};  // given dof -> padded dof
};
int launch_pad_values(const PadMap& pm, int n, int nnzb, const int* rp, const int* ci, const double* vals,
                      double* vp, cudaStream_t s);
int launch_pad_vec(const PadMap& pm, long n, const double* x, double* xp, cudaStream_t s);
int launch_unpad_vec(const PadMap& pm, long n, const double* xp, double* x, cudaStream_t s);
// one colour of sweep q of the iterated sub-solve A_ff x~ = r_f (rf: n x fb;
// first: higher colours count as zero; last: also writes x_out, see k_solve.cu)
template <typename T>
int launch_gs_inner(int b, int fb, const BgsArgs& a, const T* rf, bool first, bool last, cudaStream_t s);

// ---- colour step with the rows staged by asynchronous copies (k_staged.cu) ----
// the four-lanes-per-row colour step with every node's values, columns and
// lower-colour flags copied to shared memory ahead of use; max_row = the
// level's longest row (blocks); BAMG_EUNSUPPORTED where the layout stages
// more than the step reads (several fields, block-major values) or the slots
// exceed shared memory
template <typename T>
int launch_bgs_colour_staged(int b, int fb, const BgsArgs& a, int max_row, int* err, cudaStream_t s);
int launch_row_len_max(int n, const int* rp, int* out, cudaStream_t s);

// ---- persistent multicolour sweep (k_sweep.cu) ----
// Every colour c_lo..c_hi-1 of one field step in one launch: the colour-
// ordered node list (BgsArgs.nodes = the level's whole list) is cut into
// tiles of sweep_tile_nodes(fb) entries, numbered colour by colour
// (tile_ptr[c] = first tile of colour c); a tile waits for the tiles of its
// lower-colour neighbours (dep_lo / dep_hi [tile][colour], from sweep_plan)
// through per-tile flags.  ctrl: 4 zeroed words kept with the flags; err: the
// device error flag (kDevTimeout when a bounded wait ran out).
constexpr int kSweepMaxColours = 32;
struct SweepArgs {
    int c_lo = 0, c_hi = 0;           // colours of this field step
    int C = 0;                        // colours of the level (row length of dep_lo / dep_hi)
    const int* colour_ptr = nullptr;  // [C + 1] first position of every colour in the node list
    const int* tile_ptr = nullptr;    // [C + 1]
    const int* dep_lo = nullptr;      // [tiles][C]
    const int* dep_hi = nullptr;
    unsigned* flags = nullptr;        // [tiles]
    unsigned* ctrl = nullptr;         // ticket, exit count, epoch, spare
    int* err = nullptr;
};
int sweep_tile_nodes(int fb);  // 0: no sweep kernel for this sub-block size
// tiles = tiles of colours c_lo..c_hi-1; g4: four lanes per scalar row
template <typename T>
int launch_bgs_sweep(int b, int fb, const BgsArgs& a, const SweepArgs& sw, int tiles, int g4, cudaStream_t s);
// ---- ILU(0) sub-solve in colour order (k_ilu.cu) ----
// factors of every field's A_ff: lu[F][nnzb][fb][fb] (FP64), pos[n] receives
// each node's position in the colour-ordered list; node_field (optional)
// restricts every row to its node's field
int ilu_factor(int n, int b, int fb, int F, long nnzb, int n_colours, const std::vector<int>& colour_ptr,
               const int* nodes, const int* rp, const int* ci, const int* diag, const int* node_field,
               const double* vals, int* pos, double* lu, int* err, cudaStream_t s);
// upk[k] = 1 where block k's column has a higher colour (same node field)
int launch_upper_flags(int n, const int* rp, const int* ci, const int* colour, const int* node_field,
                       unsigned char* upk, cudaStream_t s);
// one colour of the forward (y = L^{-1} r_f, r_f formed on the fly from
// x_in, y to xt) or backward (x~ = U^{-1} y in xt, then x_out) solve of a
// field step; lu = the field's plane of factors in the cycle type
template <typename T>
int launch_ilu_colour(int b, int fb, const BgsArgs& a, const T* lu, const int* diag, const unsigned char* upk,
                      bool backward, cudaStream_t s);
// ---- restricted Schwarz sub-solve on aggregates (k_schwarz.cu) ----
struct SchwarzArgs {
    int agg_lo = 0, agg_hi = 0;  // aggregates (subdomains) of this field step
    int nfs = 1;                 // subdomains per aggregate: F (co-located fields) or 1 (node fields)
    int b = 0, fb = 0;
    const int* sd_ptr = nullptr;    // [n_agg + 1] node lists of the subdomains
    const int* sd_nodes = nullptr;
    const int* agg_ptr = nullptr;   // own nodes: the aggregate's members
    const int* members = nullptr;
    const long* x_off = nullptr;    // [n_agg * nfs + 1] offsets of the restricted inverses
    const void* X = nullptr;        // own_rows x m per subdomain, column by column (cycle type)
    const void* rf = nullptr;       // [n][fb] residual of the field
};
// node count of every subdomain (-1: more than the kernel takes)
int schwarz_setup_count(int n_agg, const int* agg_ptr, const int* members, const int* rp, const int* ci,
                        const int* node_field, int overlap, int* cnt, cudaStream_t s);
// node lists and the FP64 restricted inverses of every (aggregate, field)
int schwarz_setup_fill(int n_agg, int F, int b, int fb, int max_m, const int* agg_ptr, const int* members,
                       const int* rp, const int* ci, const int* node_field, int overlap, const int* sd_ptr,
                       int* sd_nodes, const double* vals, const long* x_off, double* X, int* err, cudaStream_t s);
// rf = rhs_f - A_{f,*} (x_in + P uc) over n rows (x_in null: rhs_f)
template <typename T>
int launch_field_residual(int b, int fb, int fm, int n, int field, const int* rp, const int* ci, const T* vals,
                          const T* x_in, const T* uc, const int* agg, const T* rhs, T* rf, cudaStream_t s);
template <typename T>
int launch_schwarz_apply(const SchwarzArgs& sa, const BgsArgs& a, cudaStream_t s);
// dependencies of every tile (tile_of: scratch of n ints)
int sweep_plan(int n, int C, int ntile, const int* nodes, const int* colour, const int* colour_ptr,
               const int* tile_ptr, const int* rp, const int* ci, const unsigned char* lowk, int n_tiles,
               int* tile_of, int* dep_lo, int* dep_hi, cudaStream_t s);
// variant 0: one thread per scalar row; 1: four lanes per scalar row, each
// taking every fourth block (the partial sums meet by shuffles)
template <typename T>
int launch_spmv_tpr(int b, int fb, int fm, int n, const int* rp, const int* ci, const T* vals, const T* x,
                    const T* rhs, T* y, cudaStream_t s, int variant = 0);
// y = (1 - omega) rhs - omega (upper-colour part of A) xt: the residual after one
// pre-smoothing sweep from zero of a one-field level with one damping value
// (xt: the sweep's x~, lowk: the lower-colour flags)
template <typename T>
int launch_residual_upper(int b, int fm, int n, const int* rp, const int* ci, const unsigned char* lowk,
                          const T* vals, const T* xt, const T* rhs, double omega, T* y, cudaStream_t s);

// One recorded step of the V-cycle below the tail level, executed by the
// cluster tail kernel (see k_solve.cu).
enum PhaseType : int {
    kPhaseBgs = 0,       // one colour of one field step: bgs
    kPhaseResidual = 1,  // y = rhs - A x: rp, ci, vals, x, rhs, y, n rows
    kPhaseRestrict = 2,  // y = R x: rp = agg_ptr, ci = members, x, y, n coarse nodes
    kPhaseGemv = 3,      // y = Ainv x: vals = FP64 inverse, x, y, n = nd
    kPhaseGemv32 = 6,    // as kPhaseGemv with the FP32 inverse
    kPhaseProlongCopy = 4,  // y = x + P rhs: ci = agg, n fine nodes
    kPhaseZero = 5,      // y = 0 over n nodes
};
struct TailPhase {
    int type;
    int n;
    BgsArgs bgs;
    const int* rp;
    const int* ci;
    const void* vals;
    const void* x;
    const void* rhs;
    void* y;
    int fm;  // residual phase: vals field-major (see vrow)
};
constexpr int kTailThreads = 512;
template <typename T>
int launch_tail(int b, int fb, const TailPhase* phases, int nphase, int cluster, cudaStream_t s);
// the same phases on every SM: a cooperative launch of grid CTAs with a grid
// barrier (bar: two zeroed words) between phases; a barrier timeout sets
// kDevTimeout in err
template <typename T>
int launch_grid_tail(int b, int fb, const TailPhase* phases, int nphase, int grid, unsigned* bar, int* err,
                     cudaStream_t s);
// CTAs of the grid tail that are resident at once on the device (0: no
// cooperative launch)
template <typename T>
int grid_tail_size(int b, int fb);
// largest resident cluster size <= want for the tail kernel (0: none)
template <typename T>
int tail_cluster_size(int b, int fb, int want);
// y = Ainv x for the dense nd x nd inverse of type S (double or float; the
// sum in S), x, y of type T
template <typename T, typename S>
int launch_dense_gemv(int nd, const S* ainv, const T* x, T* y, cudaStream_t s);
int launch_cast_d2f(long m, const double* x, float* y, cudaStream_t s);
int launch_cast_f2d(long m, const float* x, double* y, cudaStream_t s);

// ---- setup kernels (k_setup.cu) ----
// diag[i] = position of the diagonal block; flag kDevBadPattern on unsorted /
// missing diagonal / out-of-range columns
int launch_check_pattern(int n, const int* rp, const int* ci, int* diag, int* err, cudaStream_t s);
// aggregation; returns number of aggregates (>= 0) or a negative status.
// agg[n] out; agg_ptr[nc+1] and members[n] allocated by the caller after the
// count is known (second call).
struct AggWork {
    int* state;   // [n]
    int* rootid;  // [n + 1]
    int* agg1;    // [n]
    int* flag;    // [1] device
    int* host_flag;  // pinned host [1]
    unsigned char* settled = nullptr;  // [n] optional: nodes whose neighbourhood is decided
};
// d_count: 2 device ints (aggregate count, error flag); w.host_flag: 2 pinned ints
int aggregate_nodes(int n, const int* rp, const int* ci, int* agg, AggWork& w, int* d_count,
                    int* d_scan_tmp, long scan_tmp_bytes, cudaStream_t s, int* rounds_out);
int build_members(int n, int nc, const int* agg, int* agg_ptr, int* members, int* d_tmp,
                  cudaStream_t s);
// Single-CTA worklist colouring (k_setup.cu): colour[n], queues qa, qb (n ints
// each, no initial contents needed), out[0] = colour count, out[1] = 1 on
// failure (a colour above 254 or an inconsistent pattern).  Dynamic shared
// memory: 5 * n + 16 bytes.
// pre_err (optional, device): a flag that a pattern check launched before
// this kernel set to nonzero; the kernel then reads no row and reports
// failure.
constexpr int kWorklistMaxNodes = 40000;
constexpr int kWorklistSmemMax = kWorklistMaxNodes * 5 + 16;  // dynamic shared memory limit set on the kernel
__global__ void __launch_bounds__(1024) colour_worklist_kernel(int n, const int* __restrict__ rp, const int* __restrict__ ci,
                                       int* __restrict__ colour, int* __restrict__ qa, int* __restrict__ qb,
                                       int* __restrict__ out, const int* __restrict__ pre_err);
// d_queue: 2n device ints of scratch (nullptr: always use the multi-launch rounds)
int colour_nodes(int n, const int* rp, const int* ci, int* colour, int* d_flag, int* h_flag,
                 cudaStream_t s, int* n_colours, int* rounds_out, int* d_queue);
// colour_ptr[C+1] and nodes sorted by (colour, index)
int colour_order(int n, int C, const int* colour, int* colour_ptr, int* nodes, int* d_tmp,
                 cudaStream_t s);
// RAP with the tentative prolongator: symbolic (row sizes), then numeric
int rap_symbolic(int nc, const int* agg_ptr, const int* members, const int* rp, const int* ci,
                 const int* agg, int* count, int* tmp_cols, int cap, int* err, cudaStream_t s);
int rap_fill_cols(int nc, const int* rp_c, const int* tmp_cols, int cap, int* ci_c, cudaStream_t s);
int rap_numeric(int b, int nc, const int* agg_ptr, const int* members, const int* rp, const int* ci,
                const double* vals, const int* agg, const int* rp_c, const int* ci_c, double* vals_c,
                cudaStream_t s);
// per-node, per-field inverses of the diagonal blocks (FP64 in, T out)
int block_inverses(int b, int fb, int n, const int* diag, const double* vals, double* dinv64, int* err,
                   cudaStream_t s);
// dense FP64 coarsest matrix, LU with partial pivoting, inverse
int coarse_dense(int b, int n, const int* rp, const int* ci, const double* vals, double* dense,
                 cudaStream_t s);
// a (nd x nd, row-major, T = double or float) is factored in place; inv
// receives A^{-1}; piv (nd ints) receives the logical row position of every
// row; lt: nd*nd T of scratch; work: dense_lu_scratch(nd) doubles of scratch
long dense_lu_scratch(int nd);
template <typename T>
int dense_lu_inverse(int nd, T* a, int* piv, T* inv, T* lt, double* work, int* err, cudaStream_t s);

// FP32 dense LU with partial pivoting and inverse on the tensor cores
// (k_dense_tc.cu) for 0 < nd <= 2048: a (row-major nd x nd) is factored in
// place (P a = L U), inv = a^-1 (row-major), pos[r] = position of row r after
// pivoting; x: nd*nd floats of scratch, work: tc_lu_scratch_floats(nd)
// floats.  A pivot below 1e-9 ||a||_inf sets kDevSingularCoarse, a bounded
// wait that ran out kDevTimeout (in *err).
constexpr int kCoarseTcMin = 223;  // smaller coarsest matrices: the one-CTA shared-memory LU
bool tc_lu_supported(int nd);
long tc_lu_scratch_floats(int nd);
int dense_lu_inverse_tc(int nd, float* a, int* pos, float* inv, float* x, float* work, int* err, cudaStream_t s);
// C = D + sign * A B, row-major FP32 (m x k, k x n; D may be C or null) on the
// tensor cores with FP32 accuracy (three TF32 products per operand pair)
int launch_tc_gemm(int m, int n, int k, const float* A, int lda, const float* B, int ldb, const float* D, int ldd,
                   float* C, int ldc, float sign, int* err, cudaStream_t s);
int exclusive_scan(int n, const int* in, int* out, int* d_tmp, long tmp_bytes, cudaStream_t s);
long scan_tmp_bytes(int n);
int launch_convert_d2f(long m, const double* x, float* y, cudaStream_t s);

// ---- batches of independent systems (k_batched.cu) ----
// chunks of the concatenated vectors: chunk c covers [chunk_e0[c], chunk_e1[c])
// of system chunk_sys[c]; the chunks of system s are sys_chunk[s] .. sys_chunk[s+1]-1
struct SegTable {
    int nsys;
    int nchunk;
    const int* chunk_sys;
    const long* chunk_e0;
    const long* chunk_e1;
    const int* sys_chunk;
};
// out[s * ldo + v] = x_s . Y_v,s (v < nv) and x_s . x_s at v = nv when want_xx
int launch_seg_dots(const SegTable& t, const double* x, const double* Y, long ld, int nv, int want_xx,
                    double* partial, double* out, int ldo, cudaStream_t s);
// on systems with active[s] (all when active is null): x_s -= sign * sum_v h[s*ldh + v] Y_v,s; then
// mode 1: out[s*ldo + v] = x_s . Y_v,s, mode 2: out[s*ldo] = x_s . x_s, mode 0: nothing
int launch_seg_axpy_dots(const SegTable& t, double* x, const double* Y, long ld, int nv, const double* h, int ldh,
                         double sign, int mode, const int* active, double* partial, double* out, int ldo,
                         cudaStream_t s);
int launch_seg_givens(int nsys, int j, int m, const double* h1, const double* h2, const double* wsq, double* H,
                      double* cs, double* sn, double* g, double* scal, const int* incycle, cudaStream_t s);
int launch_seg_scale(const SegTable& t, const double* x, const double* scal, double* y, const int* on,
                     int check_breakdown, cudaStream_t s);
int launch_seg_init_g(int nsys, int m, const double* bsq, double* g, double* scal, cudaStream_t s);
int launch_seg_solve_upper(int nsys, int m, const int* k, const double* H, const double* g, double* y,
                           cudaStream_t s);
int batched_lu_inverse(int nsys, int b, int max_nd, const int* node_off, const long* inv_off, const int* rp,
                       const int* ci, const double* vals, double* work, double* inv, int* piv, double* col, int* err,
                       cudaStream_t s);
template <typename T>
int launch_batched_gemv(int nd_total, int b, const int* row_sys, const int* node_off, const long* inv_off,
                        const double* inv, const T* x, T* y, cudaStream_t s);
int launch_check_batch(int n, const int* rp, const int* ci, const int* node_sys, const int* node_off, int* err,
                       cudaStream_t s);
int launch_fill_sys(int nsys, const int* node_off, int scale, int* out, cudaStream_t s);
int launch_coarse_offsets(int nsys, const int* off, const int* rank, int* off_c, cudaStream_t s);

// ---- smoothed transfers and the general Galerkin product (k_transfer.cu) ----
// Row-wise product symbolic phase: count[row] distinct keys, tmp_cols[row*cap ..]
// ascending (see k_transfer.cu for the key sources); cap <= 256.
int spgemm_symbolic(int nrows, const int* xrp, const int* xci, const int* xmap, const int* yrp, const int* yci,
                    int* count, int* tmp_cols, int cap, int* err, cudaStream_t s);
int prolongator_numeric(int b, int fb, int n, const int* rp, const int* ci, const double* vals, const double* dinv,
                        const int* agg, const double* omega_p, const int* p_rp, const int* p_ci, double* p_v,
                        cudaStream_t s);
int transpose_index(int nc, const int* r_rp, const int* r_i, const int* p_rp, const int* p_ci, int* r_q, int* err,
                    cudaStream_t s);
int ap_numeric(int b, int fb, int n, const int* rp, const int* ci, const double* vals, const int* p_rp,
               const int* p_ci, const double* p_v, const int* ap_rp, const int* ap_ci, double* ap_v, cudaStream_t s);
int rap_general_numeric(int b, int fb, int nc, const int* r_rp, const int* r_i, const int* r_q, const double* p_v,
                        const int* ap_rp, const int* ap_ci, const double* ap_v, const int* rp_c, const int* ci_c,
                        double* vals_c, cudaStream_t s);
// P and R values in the cycle's storage type V (double, float, __nv_bfloat16)
template <typename V>
int transfer_values(long nnz, int F, int fb, const int* r_q, const double* p_v, V* p_out, V* r_out, cudaStream_t s);
// y (+)= M x with a field-block-diagonal M (restriction with R, prolongation with P)
template <typename T, typename V>
int launch_fdiag_spmv(int b, int fb, int nrows, const int* rp, const int* ci, const V* vals, const T* x, T* y,
                      bool add, cudaStream_t s);

// ---- learned weights (k_learned.cu) ----
int launch_features(int b, int fb, int n, const int* rp, const int* ci, const double* vals, const int* agg,
                    const int* agg_cnt, int level, float* out, int* err, cudaStream_t s);
int launch_agg_count(int n, int nc, const int* agg, int* cnt, int* err, cudaStream_t s);
int launch_agg_features(int nc, int F, const int* agg_ptr, const int* members, const float* node_feat, float* out,
                        cudaStream_t s);
int launch_pack_half(const float* p, uint16_t* p16, cudaStream_t s);
int launch_mlp_forward(const uint16_t* p16, const float* x, int n, float* y, cudaStream_t s);
size_t mlp_grad_workspace(int n);
int launch_mlp_grad(const uint16_t* p16, const float* x, const float* t, const int* head, int n, float* grad,
                    float* loss, float* work, cudaStream_t s);
int launch_adam(float* p, uint16_t* p16, const float* g, float* m, float* v, float lr, float beta1, float beta2,
                float eps, float c1, float c2, cudaStream_t s);
int launch_omega_from_mlp(int rows, int head, const float* y, double* out, int* any, cudaStream_t s);
int launch_fill(long m, double v, double* out, cudaStream_t s);

// ---- Krylov kernels (k_krylov.cu) ----
int krylov_chunks(long N);
// device pointers of the Arnoldi bookkeeping for step j of FGMRES(m)
struct GivensArgs {
    int j, m;
    const double* h1;  // projections of pass 1 (h1[j+1] = ||w||^2 before orthogonalising)
    const double* h2;  // projections of pass 2
    double* H;         // (m+1) x m Hessenberg, row-major
    double* cs;
    double* sn;
    double* g;
    double* scal;      // {h_{j+1,j}, |g_{j+1}|, breakdown, ||w|| before}
};
// out[v] = x . Y_v (v < nv) and, if want_xx, out[nv] = x . x; deterministic chunked sums
// (cond: run only where *cond is nonzero; null = always)
int launch_multi_dot(long N, const double* x, const double* Y, long ld, int nv, int want_xx, double* partial,
                     double* out, unsigned* ticket, cudaStream_t s, const unsigned* cond = nullptr);
// x -= sign * sum_v h[v] Y_v; then mode 1: out[v] = x . Y_v, mode 2: out[0] = x . x (+ Givens if ga),
// mode 3: as 2, and *reorth = 1 when ||x||^2 < 0.5 * ga.h1[j+1] (a second projection is due; its
// passes carry cond = reorth), else *reorth = 0, h2 = 0 and the Givens update; mode 0: nothing
int launch_axpy_dot(long N, double* x, const double* Y, long ld, int nv, const double* h, double sign, int mode,
                    double* partial, double* out, unsigned* ticket, const GivensArgs* ga, cudaStream_t s,
                    const unsigned* cond = nullptr, unsigned* reorth = nullptr);
int launch_solve_upper(int k, int m, const double* H, const double* g, double* y, cudaStream_t s);
int launch_scale(long N, const double* x, const double* scal, double* y, int check_breakdown, cudaStream_t s);
int launch_init_g(int m, const double* bsq, double* g, double* scal, cudaStream_t s);

}  // namespace bamg

#define BAMG_CUDA_TRY(expr)                      \
    do {                                          \
        cudaError_t _e = (expr);                  \
        if (_e != cudaSuccess) return BAMG_ECUDA; \
    } while (0)
