// Setup-phase kernels of the monolithic block AMG (Sec. 4.4 setup layouts):
// node graph checks, aggregation (Sec. 4.3.1), colouring for the multicolour
// node-block Gauss-Seidel sub-solve, the Galerkin product with the
// piecewise-constant prolongator (Sec. 3 and 4.3.1), per-field inverses of
// the node diagonal blocks, and the FP64 LU / inverse of the coarsest level.
//
// Order independence.  The aggregation and the colouring are defined by
// sequential greedy rules in ascending node order; the kernels reach the
// same result with priority rounds (a node decides once every lower-index
// node that could influence it has decided), so the result does not depend
// on thread scheduling.  A state only ever moves from "undecided" to a final
// value, so a stale read inside a round can only delay a decision.
#include "common.cuh"

namespace bamg {

// ---------------------------------------------------------------------------
// exclusive scan of int32 (3 passes: tiles, tile sums, add)
// ---------------------------------------------------------------------------
constexpr int kScanThreads = 256;
constexpr int kScanItems = 4;
constexpr int kScanTile = kScanThreads * kScanItems;

__device__ __forceinline__ int block_exclusive_scan(int v, int* total) {
    __shared__ int warp_tot[kScanThreads / kWarp];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    int x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        int y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) warp_tot[wid] = x;
    __syncthreads();
    if (wid == 0) {
        int w = lane < kScanThreads / kWarp ? warp_tot[lane] : 0;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            int y = __shfl_up_sync(0xffffffffu, w, o);
            if (lane >= o) w += y;
        }
        if (lane < kScanThreads / kWarp) warp_tot[lane] = w;
    }
    __syncthreads();
    int base = wid > 0 ? warp_tot[wid - 1] : 0;
    *total = warp_tot[kScanThreads / kWarp - 1];
    __syncthreads();
    return base + x - v;
}

__global__ void scan_tiles_kernel(int n, const int* __restrict__ in, int* __restrict__ out,
                                  int* __restrict__ tile_sums) {
    const long base = (long)blockIdx.x * kScanTile + threadIdx.x * kScanItems;
    int v[kScanItems];
    int s = 0;
#pragma unroll
    for (int t = 0; t < kScanItems; ++t) {
        v[t] = (base + t < n) ? in[base + t] : 0;
        s += v[t];
    }
    int tot;
    int ex = block_exclusive_scan(s, &tot);
#pragma unroll
    for (int t = 0; t < kScanItems; ++t) {
        if (base + t < n) out[base + t] = ex;
        ex += v[t];
    }
    if (threadIdx.x == 0) tile_sums[blockIdx.x] = tot;
}

// one CTA scans the tile sums in chunks; tile_sums[ntiles] receives the total
__global__ void scan_sums_kernel(int ntiles, int* __restrict__ tile_sums) {
    int carry = 0;
    for (int c0 = 0; c0 < ntiles; c0 += kScanThreads) {
        int idx = c0 + threadIdx.x;
        int v = idx < ntiles ? tile_sums[idx] : 0;
        int tot;
        int ex = block_exclusive_scan(v, &tot);
        if (idx < ntiles) tile_sums[idx] = carry + ex;
        carry += tot;
    }
    if (threadIdx.x == 0) tile_sums[ntiles] = carry;
}

__global__ void scan_add_kernel(int n, int* __restrict__ out, const int* __restrict__ tile_sums) {
    const long base = (long)blockIdx.x * kScanTile + threadIdx.x * kScanItems;
    const int add = tile_sums[blockIdx.x];
#pragma unroll
    for (int t = 0; t < kScanItems; ++t)
        if (base + t < n) out[base + t] += add;
}

long scan_tmp_bytes(int n) { return (long)sizeof(int) * (ceil_div(n, kScanTile) + 1); }

// out[0..n-1] = exclusive scan of in; out[n] = total (out must hold n+1 ints).
// in and out may alias.
int exclusive_scan(int n, const int* in, int* out, int* d_tmp, long tmp_bytes, cudaStream_t s) {
    const int ntiles = ceil_div(n, kScanTile);
    if (tmp_bytes < (long)sizeof(int) * (ntiles + 1)) return BAMG_EINVAL;
    if (n > 0) scan_tiles_kernel<<<ntiles, kScanThreads, 0, s>>>(n, in, out, d_tmp);
    scan_sums_kernel<<<1, kScanThreads, 0, s>>>(ntiles, d_tmp);
    if (n > 0) scan_add_kernel<<<ntiles, kScanThreads, 0, s>>>(n, out, d_tmp);
    BAMG_CUDA_TRY(cudaMemcpyAsync(out + n, d_tmp + ntiles, sizeof(int), cudaMemcpyDeviceToDevice, s));
    return launched(n > 0 ? 3 : 1);
}

// ---------------------------------------------------------------------------
// pattern checks: ascending in-range columns, diagonal present, structural
// symmetry; diag[i] = position of block (i, i)
// ---------------------------------------------------------------------------
__device__ __forceinline__ int find_col(const int* __restrict__ ci, int k0, int k1, int col) {
    while (k0 < k1) {
        int m = (k0 + k1) >> 1;
        int v = ci[m];
        if (v == col) return m;
        if (v < col) k0 = m + 1;
        else k1 = m;
    }
    return -1;
}

// Row i of a BSR pattern: row bounds inside [0, rp[n]], columns in range and
// strictly ascending, the diagonal block present, and every column j listing
// i back (structural symmetry).  diag (optional) receives the position of the
// diagonal block.  Rows of other threads are searched only inside clamped
// bounds, so a malformed pattern is reported without reading outside it.
__global__ void check_pattern_kernel(int n, const int* __restrict__ rp, const int* __restrict__ ci,
                                     int* __restrict__ diag, int* err) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int nz = rp[n];
    const int k0 = rp[i], k1 = rp[i + 1];
    int d = -1;
    if (k0 < 0 || k1 < k0 || k1 > nz) {
        set_error(err, kDevBadPattern);
        return;
    }
    for (int k = k0; k < k1; ++k) {
        int j = ci[k];
        if (j < 0 || j >= n || (k > k0 && ci[k - 1] >= j)) {
            set_error(err, kDevBadPattern);
            return;
        }
        if (j == i) d = k;
        else if (find_col(ci, min(max(rp[j], 0), nz), min(max(rp[j + 1], 0), nz), i) < 0) {
            set_error(err, kDevBadPattern);
            return;
        }
    }
    if (d < 0) set_error(err, kDevBadPattern);
    if (diag) diag[i] = d;
}

int launch_check_pattern(int n, const int* rp, const int* ci, int* diag, int* err, cudaStream_t s) {
    if (n <= 0) return BAMG_OK;
    check_pattern_kernel<<<ceil_div(n, 256), 256, 0, s>>>(n, rp, ci, diag, err);
    return launched(1);
}

// ---------------------------------------------------------------------------
// Aggregation.  Sequential rule (ascending node order): a node whose
// neighbours and itself are all free becomes a root; it and its neighbours
// form an aggregate.  Equivalently, the roots are the lexicographically-first
// maximal set of nodes with pairwise hop distance >= 3.  Priority rounds:
// an undecided node with a root within distance 2 is out; an undecided node
// with no undecided lower-index node and no root within distance 2 is a root.
// ---------------------------------------------------------------------------
enum : int { kUndecided = 0, kRoot = 1, kOut = 2 };

// a launch with the programmatic-dependent-launch attribute (the round
// kernels of aggregation and colouring)
template <typename... KArgs, typename... Args>
static cudaError_t launch_round(void (*kernel)(KArgs...), int grid, int threads, cudaStream_t s, Args... args) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)grid);
    cfg.blockDim = dim3((unsigned)threads);
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, kernel, static_cast<KArgs>(args)...);
}
// the round kernels' grid: at most four CTAs per SM, a grid-stride loop beyond
static int round_grid(int n, int threads) { return std::max(1, std::min(ceil_div(n, threads), 152 * 4)); }



// One round in two one-hop passes over the states at the start of the round.
// Pass 1: m1[i] = smallest undecided index in {i} + N(i) (INT_MAX if none),
//         r1[i] = 1 if a root is in {i} + N(i).
// Pass 2: an undecided node with r1 set on {i} + N(i) (a root within distance
//         2) is out; one whose smallest m1 over {i} + N(i) is i itself (no
//         undecided lower node within distance 2) becomes a root.
// New roots of one round are pairwise at distance >= 3, and a node becomes a
// root exactly when every lower node within distance 2 is out: the rounds
// reach the sequential ascending-order result.
// A node with no undecided node in {i} + N(i) is settled: its m1 (none) and
// r1 (a root in N(i): no new root can appear there) never change again, so
// later rounds skip it (settled: optional, zeroed before the first round).
__device__ __forceinline__ void mis2_pass1_node(int i, const int* __restrict__ rp, const int* __restrict__ ci,
                                                const int* __restrict__ state, int* __restrict__ m1,
                                                int* __restrict__ r1, unsigned char* __restrict__ settled) {
    if (settled && settled[i]) return;
    int mn = 0x7fffffff, root = 0;
    constexpr int U = 16;  // loads of a batch in flight together
    const int k0 = rp[i], k1 = rp[i + 1];
    for (int kb = k0; kb < k1; kb += U) {  // the row contains i itself (diagonal block)
        int jj[U], sj[U];
#pragma unroll
        for (int u = 0; u < U; ++u) jj[u] = kb + u < k1 ? ci[kb + u] : -1;
#pragma unroll
        for (int u = 0; u < U; ++u) sj[u] = jj[u] >= 0 ? state[jj[u]] : kOut;
#pragma unroll
        for (int u = 0; u < U; ++u) {
            if (sj[u] == kUndecided) mn = min(mn, jj[u]);
            if (sj[u] == kRoot) root = 1;
        }
    }
    m1[i] = mn;
    r1[i] = root;
    if (settled && mn == 0x7fffffff) settled[i] = 1;
}

// the rounds run as programmatic dependent launches (each is scheduled while
// its predecessor drains and waits for it in hardware), a thread per node
// (a grid-stride loop when launched smaller)
__global__ void mis2_pass1_kernel(int n, const int* __restrict__ rp, const int* __restrict__ ci,
                                  const int* __restrict__ state, int* __restrict__ m1, int* __restrict__ r1,
                                  unsigned char* __restrict__ settled) {
    pdl_wait();
    pdl_trigger();
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
        mis2_pass1_node(i, rp, ci, state, m1, r1, settled);
}

__device__ __forceinline__ void mis2_pass2_node(int i, const int* __restrict__ rp, const int* __restrict__ ci,
                                                const int* __restrict__ m1, const int* __restrict__ r1,
                                                int* __restrict__ state, int* __restrict__ any_undecided) {
    if (state[i] != kUndecided) return;
    int mn = 0x7fffffff, root = 0;
    constexpr int U = 16;  // loads of a batch in flight together
    const int k0 = rp[i], k1 = rp[i + 1];
    for (int kb = k0; kb < k1; kb += U) {
        int jj[U], mj[U], rj[U];
#pragma unroll
        for (int u = 0; u < U; ++u) jj[u] = kb + u < k1 ? ci[kb + u] : -1;
#pragma unroll
        for (int u = 0; u < U; ++u) {
            mj[u] = jj[u] >= 0 ? m1[jj[u]] : 0x7fffffff;
            rj[u] = jj[u] >= 0 ? r1[jj[u]] : 0;
        }
#pragma unroll
        for (int u = 0; u < U; ++u) {
            mn = min(mn, mj[u]);
            root |= rj[u];
        }
    }
    if (root) state[i] = kOut;
    else if (mn == i) state[i] = kRoot;
    else *any_undecided = 1;
}

__global__ void mis2_pass2_kernel(int n, const int* __restrict__ rp, const int* __restrict__ ci,
                                  const int* __restrict__ m1, const int* __restrict__ r1, int* __restrict__ state,
                                  int* __restrict__ any_undecided) {
    pdl_wait();
    pdl_trigger();
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
        mis2_pass2_node(i, rp, ci, m1, r1, state, any_undecided);
}

__global__ void is_root_kernel(int n, const int* __restrict__ state, int* __restrict__ flag) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) flag[i] = state[i] == kRoot ? 1 : 0;
}

// phase-1 membership: a root's id, or the id of the (unique) adjacent root
__global__ void assign_phase1_kernel(int n, const int* __restrict__ rp, const int* __restrict__ ci,
                                     const int* __restrict__ state, const int* __restrict__ rootid,
                                     int* __restrict__ agg1) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    int a = -1;
    if (state[i] == kRoot) a = rootid[i];
    else
        for (int k = rp[i]; k < rp[i + 1]; ++k) {
            const int j = ci[k];
            if (state[j] == kRoot) a = rootid[j];
        }
    agg1[i] = a;
}

// every node left joins the phase-1 aggregate holding most of its neighbours
// (ties: smallest aggregate id)
__global__ void attach_kernel(int n, const int* __restrict__ rp, const int* __restrict__ ci,
                              const int* __restrict__ agg1, int* __restrict__ agg, int* err) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    if (agg1[i] >= 0) {
        agg[i] = agg1[i];
        return;
    }
    int best = -1, best_count = 0;
    for (int k = rp[i]; k < rp[i + 1]; ++k) {
        const int j = ci[k];
        if (j == i) continue;
        const int a = agg1[j];
        if (a < 0) continue;
        int count = 0;
        for (int k2 = rp[i]; k2 < rp[i + 1]; ++k2) {
            const int j2 = ci[k2];
            if (j2 != i && agg1[j2] == a) count++;
        }
        if (count > best_count || (count == best_count && a < best)) {
            best = a;
            best_count = count;
        }
    }
    if (best < 0) set_error(err, kDevBadPattern);
    agg[i] = best;
}

int aggregate_nodes(int n, const int* rp, const int* ci, int* agg, AggWork& w, int* d_count,
                    int* d_scan_tmp, long scan_tmp_b, cudaStream_t s, int* rounds_out) {
    const int threads = 256, blocks = ceil_div(n, threads);
    BAMG_CUDA_TRY(cudaMemsetAsync(w.state, 0, sizeof(int) * (size_t)n, s));
    if (w.settled) BAMG_CUDA_TRY(cudaMemsetAsync(w.settled, 0, (size_t)n, s));
    const int batch = 16;
    const long max_rounds = 4L * n + 64;
    long rounds = 0;
    for (;;) {
        for (int r = 0; r < batch; ++r) {
            if (r == batch - 1) BAMG_CUDA_TRY(cudaMemsetAsync(w.flag, 0, sizeof(int), s));
            // agg1 and rootid serve as m1 and r1 during the rounds
            BAMG_CUDA_TRY(launch_round(mis2_pass1_kernel, blocks, threads, s, n, rp, ci, w.state, w.agg1, w.rootid,
                                       w.settled));
            BAMG_CUDA_TRY(launch_round(mis2_pass2_kernel, blocks, threads, s, n, rp, ci, w.agg1, w.rootid, w.state,
                                       w.flag));
        }
        note_launch(2 * batch);
        rounds += batch;
        BAMG_CUDA_TRY(cudaMemcpyAsync(w.host_flag, w.flag, sizeof(int), cudaMemcpyDeviceToHost, s));
        BAMG_CUDA_TRY(cudaStreamSynchronize(s));
        if (*w.host_flag == 0) break;
        if (rounds > max_rounds) return BAMG_ETIMEOUT;
    }
    if (rounds_out) *rounds_out = (int)rounds;
    // ids = ranks of the roots in ascending index
    is_root_kernel<<<blocks, threads, 0, s>>>(n, w.state, w.rootid);
    int st = exclusive_scan(n, w.rootid, w.rootid, d_scan_tmp, scan_tmp_b, s);
    if (st) return st;
    assign_phase1_kernel<<<blocks, threads, 0, s>>>(n, rp, ci, w.state, w.rootid, w.agg1);
    attach_kernel<<<blocks, threads, 0, s>>>(n, rp, ci, w.agg1, agg, d_count + 1);
    note_launch(3);
    BAMG_CUDA_TRY(cudaMemcpyAsync(d_count, w.rootid + n, sizeof(int), cudaMemcpyDeviceToDevice, s));
    BAMG_CUDA_TRY(cudaMemcpyAsync(w.host_flag, d_count, 2 * sizeof(int), cudaMemcpyDeviceToHost, s));
    BAMG_CUDA_TRY(cudaStreamSynchronize(s));
    if (w.host_flag[1] != 0) return BAMG_EINVAL;
    return w.host_flag[0];
}

// ---------------------------------------------------------------------------
// members of every aggregate, ascending: count, scan, scatter, sort segments
// ---------------------------------------------------------------------------
__global__ void histogram_kernel(int n, const int* __restrict__ key, int* __restrict__ count) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) atomicAdd(count + key[i], 1);
}

__global__ void scatter_by_key_kernel(int n, const int* __restrict__ key, const int* __restrict__ ptr,
                                      int* __restrict__ fill, int* __restrict__ out) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int a = key[i];
    out[ptr[a] + atomicAdd(fill + a, 1)] = i;
}

__global__ void sort_segments_kernel(int nseg, const int* __restrict__ ptr, int* __restrict__ v) {
    const int I = blockIdx.x * blockDim.x + threadIdx.x;
    if (I >= nseg) return;
    const int a = ptr[I], b = ptr[I + 1];
    for (int p = a + 1; p < b; ++p) {
        int x = v[p], q = p - 1;
        while (q >= a && v[q] > x) {
            v[q + 1] = v[q];
            --q;
        }
        v[q + 1] = x;
    }
}

// d_tmp: >= nc + 1 + scan tmp ints
int build_members(int n, int nc, const int* agg, int* agg_ptr, int* members, int* d_tmp,
                  cudaStream_t s) {
    int* count = d_tmp;                 // nc + 1
    int* scan_tmp = d_tmp + nc + 1;     // scan tmp
    BAMG_CUDA_TRY(cudaMemsetAsync(count, 0, sizeof(int) * (size_t)(nc + 1), s));
    histogram_kernel<<<ceil_div(n, 256), 256, 0, s>>>(n, agg, count);
    int st = exclusive_scan(nc, count, agg_ptr, scan_tmp, scan_tmp_bytes(nc), s);
    if (st) return st;
    BAMG_CUDA_TRY(cudaMemsetAsync(count, 0, sizeof(int) * (size_t)(nc + 1), s));
    scatter_by_key_kernel<<<ceil_div(n, 256), 256, 0, s>>>(n, agg, agg_ptr, count, members);
    sort_segments_kernel<<<ceil_div(nc, 128), 128, 0, s>>>(nc, agg_ptr, members);
    return launched(3);
}

// ---------------------------------------------------------------------------
// Colouring: sequential first fit in ascending order = Jones-Plassmann with
// index priority: a node takes the smallest colour unused by its lower-index
// neighbours once all of them are coloured.
// ---------------------------------------------------------------------------
constexpr int kMaxColours = 128;

__device__ __forceinline__ void colour_round_node(int i, const int* __restrict__ rp, const int* __restrict__ ci,
                                                  int* colour, int* flag) {
    volatile int* col = colour;
    if (col[i] >= 0) return;
    // the row's columns and their colours U at a time: the loads of a batch
    // are independent (one round trip each instead of one per neighbour)
    constexpr int U = 16;
    unsigned long long used0 = 0ull, used1 = 0ull;  // colours 0..63, 64..127
    const int k0 = rp[i], k1 = rp[i + 1];
    for (int kb = k0; kb < k1; kb += U) {
        int jj[U], cj[U];
#pragma unroll
        for (int u = 0; u < U; ++u) jj[u] = kb + u < k1 ? ci[kb + u] : i;
#pragma unroll
        for (int u = 0; u < U; ++u) cj[u] = jj[u] < i ? col[jj[u]] : 0;
        bool lower_left = true;
#pragma unroll
        for (int u = 0; u < U; ++u) {
            if (jj[u] >= i) {  // columns ascending: no lower neighbour after this one
                lower_left = false;
                continue;
            }
            if (cj[u] < 0) {  // a lower neighbour not coloured yet: next round
                *flag = 1;
                return;
            }
            if (cj[u] < 64) used0 |= 1ull << cj[u];
            else if (cj[u] < kMaxColours) used1 |= 1ull << (cj[u] - 64);
        }
        if (!lower_left) break;
    }
    // the smallest colour not in use
    int c = used0 != ~0ull ? __ffsll((long long)~used0) - 1
                           : (used1 != ~0ull ? 64 + __ffsll((long long)~used1) - 1 : kMaxColours);
    if (c >= kMaxColours) {
        flag[1] = 1;  // too many colours
        c = kMaxColours - 1;
    }
    col[i] = c;
}

// (programmatic dependent launches as the MIS-2 rounds, over a grid of at
// most four CTAs per SM: in most rounds most nodes are coloured and return)
__global__ void colour_round_kernel(int n, const int* __restrict__ rp, const int* __restrict__ ci, int* colour,
                                    int* flag) {
    pdl_wait();
    pdl_trigger();
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
        colour_round_node(i, rp, ci, colour, flag);
}

__global__ void max_kernel(int n, const int* __restrict__ v, int* out) {
    int m = -1;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) m = max(m, v[i]);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) m = max(m, __shfl_xor_sync(0xffffffffu, m, o));
    if ((threadIdx.x & 31) == 0) atomicMax(out, m);
}

// Single-CTA Jones-Plassmann for graphs that fit in shared memory: a node is
// coloured (smallest colour unused by its lower-index neighbours) as soon as
// its count of uncoloured lower-index neighbours reaches zero; the frontier
// of such nodes advances one step per iteration.  Same result as the rounds.
// The count of node j is taken from row j and decremented from the rows of
// its lower neighbours, so the rule needs a structurally symmetric pattern.
// A pattern that is not symmetric is reported (out[1] = 1), never coloured
// silently: a count that goes below zero (a lower row lists j, row j does not
// list it back), a node coloured while one of its lower neighbours is still
// uncoloured, or a node left uncoloured at the end (row j lists a lower
// neighbour whose row does not list j).
__global__ void __launch_bounds__(1024) colour_worklist_kernel(int n, const int* __restrict__ rp,
                                                               const int* __restrict__ ci, int* __restrict__ colour,
                                                               int* __restrict__ qa, int* __restrict__ qb,
                                                               int* __restrict__ out, const int* __restrict__ pre_err) {
    extern __shared__ int smem_i[];
    int* cnt = smem_i;                                            // n
    unsigned char* col = reinterpret_cast<unsigned char*>(cnt + n);  // n
    __shared__ int qn_cur, qn_next, cmax, bad;
    const int tid = threadIdx.x;
    if (tid == 0) {
        qn_cur = 0;
        qn_next = 0;
        cmax = -1;
        bad = pre_err && *pre_err != 0;  // a pattern check ahead of this launch failed
    }
    __syncthreads();
    if (bad) {  // the rows are not read: every node uncoloured, failure reported
        for (int i = tid; i < n; i += blockDim.x) colour[i] = -1;
        if (tid == 0) {
            out[0] = 0;
            out[1] = 1;
        }
        return;
    }
    for (int i = tid; i < n; i += blockDim.x) {
        int c = 0;
        for (int k = rp[i]; k < rp[i + 1]; ++k) c += ci[k] < i;
        cnt[i] = c;
        col[i] = 255;
        if (c == 0) qa[atomicAdd(&qn_cur, 1)] = i;
    }
    __syncthreads();
    int* cur = qa;
    int* nxt = qb;
    for (int guard = 0; guard <= n; ++guard) {
        const int nc = qn_cur;
        if (nc == 0) break;
        for (int q = tid; q < nc; q += blockDim.x) {
            const int i = cur[q];
            unsigned long long used[4] = {0ull, 0ull, 0ull, 0ull};
            for (int k = rp[i]; k < rp[i + 1]; ++k) {
                const int j = ci[k];
                if (j < i) {
                    const int cj = col[j];
                    used[cj >> 6] |= 1ull << (cj & 63);
                }
            }
            int c = 0;
            while (c < 255 && (used[c >> 6] >> (c & 63) & 1ull)) ++c;
            if (c >= 255 || (used[3] >> 63 & 1ull)) bad = 1;  // colour 255 = a lower neighbour not yet coloured
            col[i] = (unsigned char)c;
            atomicMax(&cmax, c);
        }
        __syncthreads();
        for (int q = tid; q < nc; q += blockDim.x) {
            const int i = cur[q];
            for (int k = rp[i]; k < rp[i + 1]; ++k) {
                const int j = ci[k];
                if (j <= i) continue;
                const int before = atomicSub(&cnt[j], 1);
                if (before == 1) nxt[atomicAdd(&qn_next, 1)] = j;
                else if (before < 1) bad = 1;  // row j does not list i
            }
        }
        __syncthreads();
        if (tid == 0) {
            qn_cur = qn_next;
            qn_next = 0;
        }
        int* t = cur;
        cur = nxt;
        nxt = t;
        __syncthreads();
    }
    int left = 0;  // nodes this thread finds uncoloured
    for (int i = tid; i < n; i += blockDim.x) {
        left += col[i] == 255;
        colour[i] = col[i] == 255 ? -1 : col[i];
    }
    if (left) bad = 1;
    __syncthreads();
    if (tid == 0) {
        out[0] = cmax + 1;
        out[1] = bad || qn_cur != 0;
    }
}

// d_flag: 3 device ints, h_flag: 3 pinned host ints
int colour_nodes(int n, const int* rp, const int* ci, int* colour, int* d_flag, int* h_flag,
                 cudaStream_t s, int* n_colours, int* rounds_out, int* d_queue) {
    const int threads = 256, blocks = ceil_div(n, threads), rgrid = round_grid(n, threads);
    if (n <= kWorklistMaxNodes && d_queue) {
        const size_t smem = (size_t)n * 5 + 16;
        // the limit is always raised to what the largest accepted graph needs,
        // never to this call's size: amg_colour_noalloc launches the same
        // kernel after raising it once per device, and a lower limit set here
        // would make its next launch on a larger graph fail
        BAMG_CUDA_TRY(cudaFuncSetAttribute(colour_worklist_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                           kWorklistSmemMax));
        colour_worklist_kernel<<<1, 1024, smem, s>>>(n, rp, ci, colour, d_queue, d_queue + n, d_flag, nullptr);
        note_launch(1);
        BAMG_CUDA_TRY(cudaMemcpyAsync(h_flag, d_flag, 2 * sizeof(int), cudaMemcpyDeviceToHost, s));
        BAMG_CUDA_TRY(cudaStreamSynchronize(s));
        if (h_flag[1]) return BAMG_EUNSUPPORTED;
        *n_colours = h_flag[0];
        if (rounds_out) *rounds_out = 0;
        return BAMG_OK;
    }
    BAMG_CUDA_TRY(cudaMemsetAsync(colour, 0xff, sizeof(int) * (size_t)n, s));
    BAMG_CUDA_TRY(cudaMemsetAsync(d_flag, 0, 3 * sizeof(int), s));
    const int batch = 32;
    const long max_rounds = 2L * n + 64;
    long rounds = 0;
    for (;;) {
        for (int r = 0; r < batch; ++r) {
            if (r == batch - 1) BAMG_CUDA_TRY(cudaMemsetAsync(d_flag, 0, sizeof(int), s));
            BAMG_CUDA_TRY(launch_round(colour_round_kernel, rgrid, threads, s, n, rp, ci, colour, d_flag));
        }
        note_launch(batch);
        rounds += batch;
        BAMG_CUDA_TRY(cudaMemcpyAsync(h_flag, d_flag, 2 * sizeof(int), cudaMemcpyDeviceToHost, s));
        BAMG_CUDA_TRY(cudaStreamSynchronize(s));
        if (h_flag[1]) return BAMG_EUNSUPPORTED;
        if (h_flag[0] == 0) break;
        if (rounds > max_rounds) return BAMG_ETIMEOUT;
    }
    if (rounds_out) *rounds_out = (int)rounds;
    BAMG_CUDA_TRY(cudaMemsetAsync(d_flag + 2, 0xff, sizeof(int), s));
    max_kernel<<<min(ceil_div(n, 256), 1024), 256, 0, s>>>(n, colour, d_flag + 2);
    note_launch(1);
    BAMG_CUDA_TRY(cudaMemcpyAsync(h_flag + 2, d_flag + 2, sizeof(int), cudaMemcpyDeviceToHost, s));
    BAMG_CUDA_TRY(cudaStreamSynchronize(s));
    *n_colours = h_flag[2] + 1;
    return BAMG_OK;
}

// nodes ordered by (colour, index): one stable compaction per colour
__global__ void eq_flag_kernel(int n, const int* __restrict__ v, int c, int* __restrict__ flag) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) flag[i] = v[i] == c ? 1 : 0;
}
__global__ void compact_kernel(int n, const int* __restrict__ v, int c, const int* __restrict__ pos,
                               const int* __restrict__ base, int* __restrict__ out) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n && v[i] == c) out[*base + pos[i]] = i;
}
__global__ void advance_kernel(int* __restrict__ colour_ptr, int c, const int* __restrict__ pos, int n) {
    colour_ptr[c + 1] = colour_ptr[c] + pos[n];
}

// d_tmp: n + 1 + scan tmp ints
int colour_order(int n, int C, const int* colour, int* colour_ptr, int* nodes, int* d_tmp,
                 cudaStream_t s) {
    int* pos = d_tmp;
    int* scan_tmp = d_tmp + n + 1;
    BAMG_CUDA_TRY(cudaMemsetAsync(colour_ptr, 0, sizeof(int), s));
    for (int c = 0; c < C; ++c) {
        eq_flag_kernel<<<ceil_div(n, 256), 256, 0, s>>>(n, colour, c, pos);
        int st = exclusive_scan(n, pos, pos, scan_tmp, scan_tmp_bytes(n), s);
        if (st) return st;
        compact_kernel<<<ceil_div(n, 256), 256, 0, s>>>(n, colour, c, pos, colour_ptr + c, nodes);
        advance_kernel<<<1, 1, 0, s>>>(colour_ptr, c, pos, n);
    }
    return launched(3 * C);
}

// ---------------------------------------------------------------------------
// Galerkin product with the tentative prolongator, one warp per coarse row I:
//   pattern: the distinct agg(j) over all stored (i, j) with agg(i) = I,
//   values:  A_c[I, J] = sum over members i of I (ascending), then over the
//            stored blocks of row i (stored order), of A[i, j] with agg(j)=J.
// The numeric pass adds the blocks one at a time in exactly that order, so
// each coarse entry is the same sequence of FP64 additions as its definition.
// ---------------------------------------------------------------------------
constexpr int kRapWarps = 4;

__global__ void __launch_bounds__(kRapWarps * 32)
    rap_symbolic_kernel(int nc, const int* __restrict__ agg_ptr, const int* __restrict__ members,
                        const int* __restrict__ rp, const int* __restrict__ ci,
                        const int* __restrict__ agg, int* __restrict__ count,
                        int* __restrict__ tmp_cols, int cap, int* err) {
    extern __shared__ int sh[];
    const int wid = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int I = blockIdx.x * kRapWarps + wid;
    if (I >= nc) return;
    int* set = sh + wid * cap;
    int size = 0;  // identical in every lane of the warp
    bool overflow = false;
    for (int q = agg_ptr[I]; q < agg_ptr[I + 1] && !overflow; ++q) {
        const int i = members[q];
        const int k0 = rp[i], k1 = rp[i + 1];
        for (int kb = k0; kb < k1 && !overflow; kb += 32) {
            const int k = kb + lane;
            const bool valid = k < k1;
            const int J = valid ? agg[ci[k]] : -1;
            bool present = !valid;
            for (int p = 0; p < size && !present; ++p) present = set[p] == J;
            const unsigned same = __match_any_sync(0xffffffffu, J);
            const bool leader = (__ffs(same) - 1) == lane;
            const unsigned fresh = __ballot_sync(0xffffffffu, leader && !present);
            const int rank = __popc(fresh & ((1u << lane) - 1u));
            const int grown = size + __popc(fresh);
            if (grown > cap) {
                overflow = true;  // uniform: every lane sees the same ballot
            } else {
                if (leader && !present) set[size + rank] = J;
                size = grown;
            }
            __syncwarp();
        }
    }
    if (overflow) {
        if (lane == 0) set_error(err, kDevRowTooLong);
        if (lane == 0) count[I] = 0;
        return;
    }
    if (lane == 0) {
        for (int p = 1; p < size; ++p) {  // insertion sort of the (short) row
            int x = set[p], r = p - 1;
            while (r >= 0 && set[r] > x) {
                set[r + 1] = set[r];
                --r;
            }
            set[r + 1] = x;
        }
        count[I] = size;
    }
    __syncwarp();
    for (int p = lane; p < size; p += 32) tmp_cols[(size_t)I * cap + p] = set[p];
}

int rap_symbolic(int nc, const int* agg_ptr, const int* members, const int* rp, const int* ci,
                 const int* agg, int* count, int* tmp_cols, int cap, int* err, cudaStream_t s) {
    if (nc <= 0) return BAMG_OK;
    const size_t smem = sizeof(int) * (size_t)cap * kRapWarps;
    rap_symbolic_kernel<<<ceil_div(nc, kRapWarps), kRapWarps * 32, smem, s>>>(
        nc, agg_ptr, members, rp, ci, agg, count, tmp_cols, cap, err);
    return launched(1);
}

__global__ void rap_fill_cols_kernel(int nc, const int* __restrict__ rp_c, const int* __restrict__ tmp,
                                     int cap, int* __restrict__ ci_c) {
    const int I = (int)(((long)blockIdx.x * blockDim.x + threadIdx.x) >> 5);
    const int lane = threadIdx.x & 31;
    if (I >= nc) return;
    for (int p = rp_c[I] + lane; p < rp_c[I + 1]; p += 32) ci_c[p] = tmp[(size_t)I * cap + (p - rp_c[I])];
}

int rap_fill_cols(int nc, const int* rp_c, const int* tmp_cols, int cap, int* ci_c, cudaStream_t s) {
    if (nc <= 0) return BAMG_OK;
    rap_fill_cols_kernel<<<ceil_div((long)nc * 32, 256), 256, 0, s>>>(nc, rp_c, tmp_cols, cap, ci_c);
    return launched(1);
}

__global__ void __launch_bounds__(kRapWarps * 32)
    rap_numeric_kernel(int b, int nc, const int* __restrict__ agg_ptr, const int* __restrict__ members,
                       const int* __restrict__ rp, const int* __restrict__ ci,
                       const double* __restrict__ vals, const int* __restrict__ agg,
                       const int* __restrict__ rp_c, const int* __restrict__ ci_c,
                       double* __restrict__ vals_c) {
    const int wid = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int I = blockIdx.x * kRapWarps + wid;
    if (I >= nc) return;
    const int bb = b * b;
    const int c0 = rp_c[I], c1 = rp_c[I + 1];
    double* out = vals_c + (size_t)c0 * bb;
    for (int e = lane; e < (c1 - c0) * bb; e += 32) out[e] = 0.0;
    __syncwarp();
    for (int q = agg_ptr[I]; q < agg_ptr[I + 1]; ++q) {
        const int i = members[q];
        for (int k = rp[i]; k < rp[i + 1]; ++k) {
            const int J = agg[ci[k]];
            int lo = c0, hi = c1;  // binary search of J in the sorted coarse row
            while (lo < hi) {
                int m = (lo + hi) >> 1;
                if (ci_c[m] < J) lo = m + 1;
                else hi = m;
            }
            double* dst = vals_c + (size_t)lo * bb;
            const double* src = vals + (size_t)k * bb;
            for (int e = lane; e < bb; e += 32) dst[e] = __dadd_rn(dst[e], src[e]);
        }
    }
}

int rap_numeric(int b, int nc, const int* agg_ptr, const int* members, const int* rp, const int* ci,
                const double* vals, const int* agg, const int* rp_c, const int* ci_c, double* vals_c,
                cudaStream_t s) {
    if (nc <= 0) return BAMG_OK;
    rap_numeric_kernel<<<ceil_div(nc, kRapWarps), kRapWarps * 32, 0, s>>>(b, nc, agg_ptr, members, rp, ci,
                                                                        vals, agg, rp_c, ci_c, vals_c);
    return launched(1);
}

// ---------------------------------------------------------------------------
// per-node, per-field inverses of the diagonal blocks: Gauss-Jordan with
// partial pivoting (first maximum wins); singular when a pivot magnitude is
// below 1e-14 * (infinity norm of the block)
// ---------------------------------------------------------------------------
template <int FB>
__global__ void block_inverse_kernel(int b, int F, int n, const int* __restrict__ diag,
                                     const double* __restrict__ vals, double* __restrict__ dinv, int* err) {
    const long t = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= (long)n * F) return;
    const int i = (int)(t / F), f = (int)(t - (long)i * F);
    const double* blk = vals + (size_t)diag[i] * b * b;
    double w[FB][FB], v[FB][FB];
    double norm = 0.0;
#pragma unroll
    for (int r = 0; r < FB; ++r) {
        double sum = 0.0;
#pragma unroll
        for (int c = 0; c < FB; ++c) {
            w[r][c] = blk[(f * FB + r) * b + f * FB + c];
            v[r][c] = (r == c) ? 1.0 : 0.0;
            sum += fabs(w[r][c]);
        }
        norm = fmax(norm, sum);
    }
    bool singular = norm == 0.0;
#pragma unroll
    for (int k = 0; k < FB; ++k) {
        int p = k;
#pragma unroll
        for (int r = k + 1; r < FB; ++r)
            if (fabs(w[r][k]) > fabs(w[p][k])) p = r;
        if (!(fabs(w[p][k]) >= 1e-14 * norm)) singular = true;
        // swap rows k and p (register arrays: select by predicate)
#pragma unroll
        for (int r = k + 1; r < FB; ++r) {
            if (r == p) {
#pragma unroll
                for (int c = 0; c < FB; ++c) {
                    double tw = w[k][c];
                    w[k][c] = w[r][c];
                    w[r][c] = tw;
                    double tv = v[k][c];
                    v[k][c] = v[r][c];
                    v[r][c] = tv;
                }
            }
        }
        const double piv = w[k][k];
#pragma unroll
        for (int c = 0; c < FB; ++c) {
            w[k][c] = __ddiv_rn(w[k][c], piv);
            v[k][c] = __ddiv_rn(v[k][c], piv);
        }
#pragma unroll
        for (int r = 0; r < FB; ++r) {
            if (r == k) continue;
            const double fr = w[r][k];
#pragma unroll
            for (int c = 0; c < FB; ++c) {
                w[r][c] = __dsub_rn(w[r][c], __dmul_rn(fr, w[k][c]));
                v[r][c] = __dsub_rn(v[r][c], __dmul_rn(fr, v[k][c]));
            }
        }
    }
    if (singular) set_error(err, kDevSingularBlock);
    double* out = dinv + (size_t)t * FB * FB;
#pragma unroll
    for (int r = 0; r < FB; ++r)
#pragma unroll
        for (int c = 0; c < FB; ++c) out[r * FB + c] = v[r][c];
}

int block_inverses(int b, int fb, int n, const int* diag, const double* vals, double* dinv64, int* err,
                   cudaStream_t s) {
    const int F = b / fb;
    const int blocks = ceil_div((long)n * F, 128);
    if (n <= 0) return BAMG_OK;
    switch (fb) {
#define CASE(FF) \
    case FF: block_inverse_kernel<FF><<<blocks, 128, 0, s>>>(b, F, n, diag, vals, dinv64, err); break;
        CASE(1) CASE(2) CASE(3) CASE(4) CASE(5) CASE(6) CASE(7) CASE(8)
#undef CASE
        default: return BAMG_EUNSUPPORTED;
    }
    return launched(1);
}

// ---------------------------------------------------------------------------
// coarsest level: dense FP64 copy, LU with partial pivoting (first maximum
// wins; multiplier l = a[r][k] / a[k][k], update a[r][c] -= l * a[k][c] as a
// rounded product then a rounded difference, no fused multiply-add), then
// the inverse from L U X = P.
// ---------------------------------------------------------------------------
__global__ void coarse_dense_kernel(int b, int n, const int* __restrict__ rp, const int* __restrict__ ci,
                                    const double* __restrict__ vals, double* __restrict__ dense) {
    const int i = blockIdx.x;
    const int nd = n * b;
    for (int k = rp[i]; k < rp[i + 1]; ++k) {
        const int j = ci[k];
        for (int e = threadIdx.x; e < b * b; e += blockDim.x) {
            const int r = e / b, c = e - r * b;
            dense[(size_t)(i * b + r) * nd + j * b + c] = vals[(size_t)k * b * b + e];
        }
    }
}

int coarse_dense(int b, int n, const int* rp, const int* ci, const double* vals, double* dense,
                 cudaStream_t s) {
    const long nd = (long)n * b;
    BAMG_CUDA_TRY(cudaMemsetAsync(dense, 0, sizeof(double) * nd * nd, s));
    coarse_dense_kernel<<<n, 64, 0, s>>>(b, n, rp, ci, vals, dense);
    return launched(1);
}

// LU factorisation.  Small nd: one CTA factors the matrix held in shared
// memory; larger: one cooperative launch (below), else one pivot kernel and
// one rank-1 update kernel per column.  All perform the same rounded
// operations in the same order per entry, so the factors do not depend on
// the variant.  T = double is the coarse solve of the method; T = float
// factors the FP32 copy of the coarsest matrix for FP32 cycles (GB300 issues
// FP32 at 64 times its FP64 rate).
constexpr int kLuThreads = 1024;
// largest nd whose nd^2 entries fit 199.7 KB of shared memory (158^2 doubles)
template <typename T>
struct LuSmem {
    static constexpr int kMax = sizeof(T) == 8 ? 158 : 223;
};
// a smallest pivot of 1e-14 (FP64) or 1e-9 (FP32) times the infinity norm
// marks the matrix singular.  (In FP32 pivots between that and the rounding
// level leave the coarse solve inaccurate along near-null directions, which
// the outer FGMRES absorbs: the stabilised 3D Stokes coarsest operator has
// such a pivot and converges in the same iterations as with the FP64 solve.)
template <typename T>
__host__ __device__ constexpr T lu_tiny() {
    return sizeof(T) == 8 ? T(1e-14) : T(1e-9);
}

// correctly rounded single operations (no contraction into fused multiply-adds)
__device__ __forceinline__ double rn_div(double a, double b) { return __ddiv_rn(a, b); }
__device__ __forceinline__ float rn_div(float a, float b) { return __fdiv_rn(a, b); }
__device__ __forceinline__ double rn_mul(double a, double b) { return __dmul_rn(a, b); }
__device__ __forceinline__ float rn_mul(float a, float b) { return __fmul_rn(a, b); }
__device__ __forceinline__ double rn_sub(double a, double b) { return __dsub_rn(a, b); }
__device__ __forceinline__ float rn_sub(float a, float b) { return __fsub_rn(a, b); }

// first row r >= k of maximal |a[r][k]| over the CTA (ties: smallest r)
template <typename T>
__device__ __forceinline__ void pivot_search(const T* a, int nd, int k, T* red_v, int* red_i, T* best_out,
                                             int* idx_out) {
    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
    T best = T(-1);
    int bi = nd;
    for (int r = k + tid; r < nd; r += blockDim.x) {
        const T v = fabs(a[(size_t)r * nd + k]);
        if (v > best) {
            best = v;
            bi = r;
        }
    }
    for (int o = 16; o > 0; o >>= 1) {
        const T ov = __shfl_xor_sync(0xffffffffu, best, o);
        const int oi = __shfl_xor_sync(0xffffffffu, bi, o);
        if (ov > best || (ov == best && oi < bi)) {
            best = ov;
            bi = oi;
        }
    }
    if (lane == 0) {
        red_v[wid] = best;
        red_i[wid] = bi;
    }
    __syncthreads();
    if (tid == 0) {
        T bv = red_v[0];
        int bx = red_i[0];
        for (int w = 1; w < (int)(blockDim.x / 32); ++w)
            if (red_v[w] > bv || (red_v[w] == bv && red_i[w] < bx)) {
                bv = red_v[w];
                bx = red_i[w];
            }
        red_v[0] = bv;
        red_i[0] = bx;
    }
    __syncthreads();
    *best_out = red_v[0];
    *idx_out = red_i[0];
    __syncthreads();
}

// infinity norm (largest absolute row sum) of the nd x nd matrix a
template <typename T>
__device__ __forceinline__ T inf_norm(const T* a, int nd, T* red_v) {
    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
    T m = T(0);
    for (int r = tid; r < nd; r += blockDim.x) {
        T sum = T(0);
        for (int c = 0; c < nd; ++c) sum += fabs(a[(size_t)r * nd + c]);
        m = fmax(m, sum);
    }
    for (int o = 16; o > 0; o >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, o));
    if (lane == 0) red_v[wid] = m;
    __syncthreads();
    T mm = T(0);
    for (int w = 0; w < (int)(blockDim.x / 32); ++w) mm = fmax(mm, red_v[w]);
    __syncthreads();
    return mm;
}

template <typename T>
__global__ void __launch_bounds__(kLuThreads) lu_smem_kernel(int nd, T* __restrict__ g, int* __restrict__ piv,
                                                             int* err) {
    extern __shared__ __align__(16) unsigned char lu_sh[];
    T* sa = reinterpret_cast<T*>(lu_sh);
    __shared__ T red_v[kLuThreads / 32];
    __shared__ int red_i[kLuThreads / 32];
    __shared__ T col[LuSmem<T>::kMax];
    const int tid = threadIdx.x;
    for (int e = tid; e < nd * nd; e += blockDim.x) sa[e] = g[e];
    __syncthreads();
    const T norm = inf_norm(sa, nd, red_v);
    bool singular = norm == T(0);
    for (int k = 0; k < nd; ++k) {
        T best;
        int p;
        pivot_search(sa, nd, k, red_v, red_i, &best, &p);
        if (!(best >= lu_tiny<T>() * norm)) singular = true;
        if (tid == 0) piv[k] = p;
        if (p != k)
            for (int c = tid; c < nd; c += blockDim.x) {
                const T t = sa[k * nd + c];
                sa[k * nd + c] = sa[p * nd + c];
                sa[p * nd + c] = t;
            }
        __syncthreads();
        const T akk = sa[k * nd + k];
        for (int r = k + 1 + tid; r < nd; r += blockDim.x) col[r] = rn_div(sa[r * nd + k], akk);
        __syncthreads();
        const int m = nd - k - 1;
        for (int e = tid; e < m * m; e += blockDim.x) {
            const int r = k + 1 + e / m, c = k + 1 + e % m;
            sa[r * nd + c] = rn_sub(sa[r * nd + c], rn_mul(col[r], sa[k * nd + c]));
        }
        for (int r = k + 1 + tid; r < nd; r += blockDim.x) sa[r * nd + k] = col[r];
        __syncthreads();
    }
    if (singular && tid == 0) set_error(err, kDevSingularCoarse);
    for (int e = tid; e < nd * nd; e += blockDim.x) g[e] = sa[e];
}

// infinity norm over the grid: one warp per row (coalesced), the row maxima
// combined by an atomic maximum on the bit patterns (non-negative values
// order like their bits); *norm_out must be zero before the launch
__device__ __forceinline__ void atomic_max_nonneg(double* p, double v) {
    atomicMax(reinterpret_cast<unsigned long long*>(p), (unsigned long long)__double_as_longlong(v));
}
__device__ __forceinline__ void atomic_max_nonneg(float* p, float v) {
    atomicMax(reinterpret_cast<unsigned*>(p), __float_as_uint(v));
}
template <typename T>
__global__ void lu_norm_rows_kernel(int nd, const T* __restrict__ a, T* __restrict__ norm_out) {
    const long r = ((long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (r >= nd) return;
    T sum = T(0);
    for (int c = lane; c < nd; c += 32) sum += fabs(a[(size_t)r * nd + c]);
    sum = warp_sum(sum);
    if (lane == 0) atomic_max_nonneg(norm_out, sum);
}

// column k: pivot, row swap, multipliers (stored in column k and in col)
template <typename T>
__global__ void __launch_bounds__(kLuThreads) lu_pivot_kernel(int nd, int k, T* __restrict__ a,
                                                              int* __restrict__ piv, T* __restrict__ col,
                                                              const T* __restrict__ norm, int* err) {
    __shared__ T red_v[kLuThreads / 32];
    __shared__ int red_i[kLuThreads / 32];
    const int tid = threadIdx.x;
    T best;
    int p;
    pivot_search(a, nd, k, red_v, red_i, &best, &p);
    if (tid == 0) {
        piv[k] = p;
        if (!(best >= lu_tiny<T>() * norm[0]) || norm[0] == T(0)) set_error(err, kDevSingularCoarse);
    }
    if (p != k)
        for (int c = tid; c < nd; c += blockDim.x) {
            const T t = a[(size_t)k * nd + c];
            a[(size_t)k * nd + c] = a[(size_t)p * nd + c];
            a[(size_t)p * nd + c] = t;
        }
    __syncthreads();
    const T akk = a[(size_t)k * nd + k];
    for (int r = k + 1 + tid; r < nd; r += blockDim.x) {
        const T l = rn_div(a[(size_t)r * nd + k], akk);
        col[r] = l;
        a[(size_t)r * nd + k] = l;
    }
}

// trailing update a[r][c] -= col[r] * a[k][c] for r, c > k
template <typename T>
__global__ void lu_update_kernel(int nd, int k, T* __restrict__ a, const T* __restrict__ col) {
    const int m = nd - k - 1;
    const long total = (long)m * m;
    for (long e = (long)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (long)gridDim.x * blockDim.x) {
        const int r = k + 1 + (int)(e / m), c = k + 1 + (int)(e % m);
        a[(size_t)r * nd + c] = rn_sub(a[(size_t)r * nd + c], rn_mul(col[r], a[(size_t)k * nd + c]));
    }
}

// lt = transpose of the packed LU factors (column k of L and U contiguous);
// logical row r of the factors is row perm[r] of a
template <typename T>
__global__ void transpose_kernel(int nd, const T* __restrict__ a, const int* __restrict__ perm, T* __restrict__ lt) {
    __shared__ T tile[32][33];
    const int bx = blockIdx.x * 32, by = blockIdx.y * 32;
    for (int y = threadIdx.y; y < 32; y += blockDim.y) {
        const int r = by + y, c = bx + threadIdx.x;
        if (r < nd && c < nd) tile[y][threadIdx.x] = a[(size_t)perm[r] * nd + c];
    }
    __syncthreads();
    for (int y = threadIdx.y; y < 32; y += blockDim.y) {
        const int r = bx + y, c = by + threadIdx.x;
        if (r < nd && c < nd) lt[(size_t)r * nd + c] = tile[threadIdx.x][y];
    }
}

// Inverse column by column: column c of A^{-1} solves L U x = P e_c, whose
// one sits at the logical position pos[c].  One CTA per column (grid-stride
// over columns), x in shared memory; lt holds the factors column-major so
// that the threads of a step read consecutive addresses.  (Several columns
// per CTA measured slower: the larger shared-memory share cuts the CTAs per
// SM that hide the steps' latency.)
constexpr int kInvThreads = 256;
// NC columns per CTA: each step's factor column is loaded once for all of them
// (FP32: two columns put the 2048 columns of the 3D coarsest level in one
// wave of resident CTAs); the operations per column are those of NC = 1
template <typename T, int NC>
__global__ void __launch_bounds__(kInvThreads) lu_inverse_cols_kernel(int nd, const T* __restrict__ lt,
                                                                      const int* __restrict__ pos,
                                                                      T* __restrict__ inv) {
    extern __shared__ __align__(16) unsigned char inv_sh[];
    T* x = reinterpret_cast<T*>(inv_sh);  // [NC][nd]
    __shared__ int pos0[NC];
    __shared__ int kmin;
    const int tid = threadIdx.x;
    for (int c0 = blockIdx.x * NC; c0 < nd; c0 += gridDim.x * NC) {
        if (tid < NC) pos0[tid] = c0 + tid < nd ? pos[c0 + tid] : nd;
        for (int r = tid; r < NC * nd; r += blockDim.x) x[r] = T(0);
        __syncthreads();
        if (tid == 0) {
            int m = nd;
            for (int j = 0; j < NC; ++j) {
                if (pos0[j] < nd) x[(size_t)j * nd + pos0[j]] = T(1);
                m = min(m, pos0[j]);
            }
            kmin = m;
        }
        __syncthreads();
        for (int k = kmin; k < nd; ++k) {  // unit lower triangle (entries above pos0 stay zero)
            T xk[NC];
            bool any = false;
#pragma unroll
            for (int j = 0; j < NC; ++j) {
                xk[j] = x[(size_t)j * nd + k];
                any |= xk[j] != T(0);
            }
            if (any)
                for (int r = k + 1 + tid; r < nd; r += blockDim.x) {
                    const T l = lt[(size_t)k * nd + r];
#pragma unroll
                    for (int j = 0; j < NC; ++j)
                        if (xk[j] != T(0)) x[(size_t)j * nd + r] -= l * xk[j];
                }
            __syncthreads();
        }
        for (int k = nd - 1; k >= 0; --k) {  // upper triangle
            if (tid < NC) x[(size_t)tid * nd + k] /= lt[(size_t)k * nd + k];
            __syncthreads();
            T xk[NC];
#pragma unroll
            for (int j = 0; j < NC; ++j) xk[j] = x[(size_t)j * nd + k];
            for (int r = tid; r < k; r += blockDim.x) {
                const T u = lt[(size_t)k * nd + r];
#pragma unroll
                for (int j = 0; j < NC; ++j) x[(size_t)j * nd + r] -= u * xk[j];
            }
            __syncthreads();
        }
        for (int j = 0; j < NC; ++j)
            if (c0 + j < nd)
                for (int r = tid; r < nd; r += blockDim.x) inv[(size_t)r * nd + c0 + j] = x[(size_t)j * nd + r];
        __syncthreads();
    }
}

// Row order of factors computed with physical row swaps (the shared-memory and
// per-column paths): the factors are already in logical order (perm = the
// identity); pos[c] = where row c of A ends up after the swaps piv[0..nd).
__global__ void swaps_to_pos_kernel(int nd, const int* __restrict__ piv, int* __restrict__ perm,
                                    int* __restrict__ pos) {
    for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < nd; c += gridDim.x * blockDim.x) {
        int p = c;
        for (int k = 0; k < nd; ++k) {
            const int pk = piv[k];
            if (pk == p) p = k;
            else if (k == p) p = pk;
        }
        pos[c] = p;
        perm[c] = c;
    }
}

// ---------------------------------------------------------------------------
// LU of a larger coarsest matrix in one cooperative launch (one CTA per SM).
// The arithmetic per entry is that of the per-column path (multiplier by a
// rounded division, update as a rounded product then a rounded difference,
// columns in order), so the factors are the same bits; only the schedule
// differs:
//  * rows are never moved: every CTA keeps the same permutation perm
//    (logical -> physical row) and its inverse pos in shared memory and
//    applies each pivot swap to them;
//  * CTA q owns the physical rows q, q + G, ...; in step k it forms the
//    multipliers of its owned rows below the pivot (shared memory), then all
//    its threads sweep the columns c > k, each loading the pivot-row entry
//    once and updating it into every owned row; the thread of column k + 1
//    offers the largest |a[row][k+1]| as the pivot candidate of the next step
//    (ties: smallest logical row);
//  * one grid barrier per column separates the steps; the per-CTA
//    candidates go through a two-slot buffer (step parity), so a fast CTA
//    never overwrites candidates that a slow one still reads.
// The barrier is a counter plus a generation word in global memory; a wait
// that exceeds its bound sets kDevTimeout and the CTA returns (the others then
// run out at their next barrier), so the kernel always ends.
// ---------------------------------------------------------------------------
constexpr int kCoopThreads = 512;
constexpr int kCoopMaxCtas = 256;
// (v, i) -> the CTA's maximum v, ties to the smallest i; valid in thread 0
template <typename T>
__device__ __forceinline__ void cta_argmax(T& v, int& i, T* red_v, int* red_i) {
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    for (int o = 16; o > 0; o >>= 1) {
        const T ov = __shfl_xor_sync(0xffffffffu, v, o);
        const int oi = __shfl_xor_sync(0xffffffffu, i, o);
        if (ov > v || (ov == v && oi < i)) {
            v = ov;
            i = oi;
        }
    }
    if (lane == 0) {
        red_v[wid] = v;
        red_i[wid] = i;
    }
    __syncthreads();
    if (threadIdx.x == 0)
        for (int w = 1; w < (int)(blockDim.x >> 5); ++w)
            if (red_v[w] > v || (red_v[w] == v && red_i[w] < i)) {
                v = red_v[w];
                i = red_i[w];
            }
    __syncthreads();
}

template <typename T>
__global__ void __launch_bounds__(kCoopThreads) lu_coop_kernel(int nd, T* __restrict__ a, const T* __restrict__ norm,
                                                                T* __restrict__ cand_v, int* __restrict__ cand_i,
                                                                unsigned* __restrict__ bar, int* __restrict__ perm_out,
                                                                int* __restrict__ pos_out, int* err) {
    const int G = gridDim.x, q = blockIdx.x, tid = threadIdx.x;
    const int lane = tid & 31, warp = tid >> 5;
    const int M = (nd - q + G - 1) / G;  // owned physical rows q + G m, m < M
    extern __shared__ __align__(16) int sh_rows[];
    int* perm = sh_rows;                 // [nd] logical -> physical
    int* pos = sh_rows + nd;             // [nd] physical -> logical
    int* s_act = sh_rows + 2 * nd;       // [M] 1 if the owned row is below the pivot
    T* s_l = reinterpret_cast<T*>(sh_rows + 2 * nd + ((M + 1) & ~1));  // [M] multipliers
    __shared__ T red_v[kCoopThreads / 32];
    __shared__ int red_i[kCoopThreads / 32];
    __shared__ int s_piv;
    for (int r = tid; r < nd; r += blockDim.x) {
        perm[r] = r;
        pos[r] = r;
    }
    // candidates for column 0: the owned rows
    T bv = T(-1);
    int bi = nd;
    for (int m = tid; m < M; m += blockDim.x) {
        const int ph = q + G * m;
        const T v = fabs(__ldcg(a + (size_t)ph * nd));
        if (v > bv || (v == bv && ph < bi)) {
            bv = v;
            bi = ph;
        }
    }
    cta_argmax(bv, bi, red_v, red_i);
    if (tid == 0) {
        cand_v[q] = bv;
        cand_i[q] = bi;
    }
    if (!grid_barrier(bar, err)) return;
    for (int k = 0; k < nd; ++k) {
        const int buf = (k & 1) * G;
        if (warp == 0) {  // the pivot of column k from the G candidates
            T v = T(-1);
            int i = nd;
            for (int c = lane; c < G; c += 32) {
                const T cv = __ldcg(cand_v + buf + c);
                const int ci = __ldcg(cand_i + buf + c);
                if (cv > v || (cv == v && ci < i)) {
                    v = cv;
                    i = ci;
                }
            }
            for (int o = 16; o > 0; o >>= 1) {
                const T ov = __shfl_xor_sync(0xffffffffu, v, o);
                const int oi = __shfl_xor_sync(0xffffffffu, i, o);
                if (ov > v || (ov == v && oi < i)) {
                    v = ov;
                    i = oi;
                }
            }
            if (lane == 0) {
                s_piv = i;
                const int pk = perm[k], pp = perm[i];
                perm[k] = pp;
                perm[i] = pk;
                pos[pp] = k;
                pos[pk] = i;
                if (q == 0 && (!(v >= lu_tiny<T>() * norm[0]) || norm[0] == T(0)))
                    set_error(err, kDevSingularCoarse);
            }
        }
        __syncthreads();
        const int pr = perm[k];
        const T* prow = a + (size_t)pr * nd;
        const T akk = __ldcg(prow + k);
        // multipliers of the owned rows below the pivot (stored in column k)
        for (int m = tid; m < M; m += blockDim.x) {
            const int ph = q + G * m;
            const int act = pos[ph] > k;
            s_act[m] = act;
            if (act) {
                const T l = rn_div(__ldcg(a + (size_t)ph * nd + k), akk);
                s_l[m] = l;
                a[(size_t)ph * nd + k] = l;
            }
        }
        __syncthreads();
        // trailing update of the owned rows; thread 0 holds column k + 1
        // (loading every owned row's entry before the stores measured slower:
        // the register tile lowers the occupancy more than it overlaps loads)
        bv = T(-1);
        bi = nd;
        for (int c = k + 1 + tid; c < nd; c += blockDim.x) {
            const T pc = __ldcg(prow + c);
            for (int m = 0; m < M; ++m) {
                if (!s_act[m]) continue;
                T* e = a + (size_t)(q + G * m) * nd + c;
                const T v = rn_sub(__ldcg(e), rn_mul(s_l[m], pc));
                *e = v;
                if (c == k + 1) {
                    const int lr = pos[q + G * m];
                    const T av = fabs(v);
                    if (av > bv || (av == bv && lr < bi)) {
                        bv = av;
                        bi = lr;
                    }
                }
            }
        }
        if (tid == 0) {  // candidates of column k + 1 into the other slot
            cand_v[(G - buf) + q] = bv;
            cand_i[(G - buf) + q] = bi;
        }
        if (!grid_barrier(bar, err)) return;
    }
    if (q == 0)
        for (int r = tid; r < nd; r += blockDim.x) {
            perm_out[r] = perm[r];
            pos_out[r] = pos[r];
        }
}

// ---------------------------------------------------------------------------
// LU with every CTA's owned rows resident in its shared memory (one CTA per
// SM; CTA q owns the physical rows q, q + G, ...), for matrices whose rows
// fit.  A step then touches shared memory only, apart from the pivot row,
// which the CTA that offered it as the next candidate published before the
// barrier.  Same pivot choice and the same rounded operations per entry as
// the other paths (the factors are the same bits):
//  * s_pos[m] is the logical position of owned row m (the order the row swaps
//    of the other paths produce): step k moves the winner to k and the row
//    that sat at k to the winner's old position;
//  * each CTA's candidate for column k + 1 is its active row with the largest
//    |a[row][k+1]| (ties: smallest logical position), published with its
//    value, physical row and logical position, and its entries from column
//    k + 1 on, into slot (k + 1) & 1 (two slots: a fast CTA never overwrites
//    a row that a slow one still reads).
// ---------------------------------------------------------------------------
constexpr int kRowsThreads = 512;
constexpr int kRowsCols = 8;  // columns per thread: nd <= kRowsCols * kRowsThreads = 4096

template <typename T>
__device__ void rows_candidate(int nd, int col, int M, const T* rows, const int* s_pos, const int* s_done, T* red_v,
                               int* red_i, T* cand_v, int* cand_i, int* cand_p, T* slot) {
    __shared__ int s_m;
    __shared__ int s_li;
    __shared__ T s_v;
    const int G = gridDim.x, q = blockIdx.x;
    T v = T(-1);
    int li = nd;
    for (int m = threadIdx.x; m < M; m += blockDim.x)
        if (!s_done[m]) {
            const T av = fabs(rows[(size_t)m * nd + col]);
            const int lp = s_pos[m];
            if (av > v || (av == v && lp < li)) {
                v = av;
                li = lp;
            }
        }
    cta_argmax(v, li, red_v, red_i);
    if (threadIdx.x == 0) {
        s_v = v;
        s_li = li;
        s_m = -1;
    }
    __syncthreads();
    for (int m = threadIdx.x; m < M; m += blockDim.x)
        if (!s_done[m] && s_pos[m] == s_li) s_m = m;
    __syncthreads();
    const int mm = s_m;
    if (threadIdx.x == 0) {  // the signed value: the pivot itself when the row wins
        cand_v[q] = mm >= 0 ? rows[(size_t)mm * nd + col] : T(0);
        cand_i[q] = mm >= 0 ? q + G * mm : nd;
        cand_p[q] = mm >= 0 ? s_li : nd;
    }
    if (mm >= 0) {
        T* dst = slot + (size_t)q * nd;
        const T* src = rows + (size_t)mm * nd;
        for (int c = col + threadIdx.x; c < nd; c += blockDim.x) dst[c] = src[c];
    }
}

template <typename T>
__global__ void __launch_bounds__(kRowsThreads) lu_rows_kernel(int nd, T* __restrict__ a, const T* __restrict__ norm,
                                                                T* __restrict__ cand_v, int* __restrict__ cand_i,
                                                                int* __restrict__ cand_p, T* __restrict__ slots,
                                                                unsigned* __restrict__ bar, int* __restrict__ perm_out,
                                                                int* __restrict__ pos_out, int* err) {
    const int G = gridDim.x, q = blockIdx.x, tid = threadIdx.x;
    const int lane = tid & 31, warp = tid >> 5;
    const int M = (nd - q + G - 1) / G;  // owned rows q + G m, m < M
    const int Mmax = (nd + G - 1) / G;
    extern __shared__ __align__(16) unsigned char rows_sh[];
    T* rows = reinterpret_cast<T*>(rows_sh);       // [Mmax][nd]
    T* s_l = rows + (size_t)Mmax * nd;             // [Mmax] multipliers
    int* s_pos = reinterpret_cast<int*>(s_l + Mmax);  // [Mmax] logical positions
    int* s_done = s_pos + Mmax;                    // [Mmax] 1 once the row was a pivot
    __shared__ T red_v[kRowsThreads / 32];
    __shared__ int red_i[kRowsThreads / 32];
    __shared__ int s_w, s_lw, s_qw;
    __shared__ T s_akk;
    for (int m = 0; m < M; ++m)
        for (int c = tid; c < nd; c += blockDim.x) rows[(size_t)m * nd + c] = __ldcg(a + (size_t)(q + G * m) * nd + c);
    for (int m = tid; m < M; m += blockDim.x) {
        s_pos[m] = q + G * m;
        s_done[m] = 0;
    }
    __syncthreads();
    const size_t slot_sz = (size_t)G * nd;
    rows_candidate(nd, 0, M, rows, s_pos, s_done, red_v, red_i, cand_v, cand_i, cand_p, slots);
    if (!grid_barrier(bar, err)) return;
    for (int k = 0; k < nd; ++k) {
        const int par = k & 1;
        if (warp == 0) {  // the pivot of column k from the G candidates
            T v = T(-1);
            int li = nd, qw = 0;
            for (int c = lane; c < G; c += 32) {
                const int cp = __ldcg(cand_p + par * G + c);
                const T cv = cp < nd ? fabs(__ldcg(cand_v + par * G + c)) : T(-1);  // nd: no active row
                if (cv > v || (cv == v && cp < li)) {
                    v = cv;
                    li = cp;
                    qw = c;
                }
            }
            for (int o = 16; o > 0; o >>= 1) {
                const T ov = __shfl_xor_sync(0xffffffffu, v, o);
                const int ol = __shfl_xor_sync(0xffffffffu, li, o);
                const int oq = __shfl_xor_sync(0xffffffffu, qw, o);
                if (ov > v || (ov == v && ol < li)) {
                    v = ov;
                    li = ol;
                    qw = oq;
                }
            }
            if (lane == 0) {
                s_lw = li;
                s_qw = qw;
                s_w = __ldcg(cand_i + par * G + qw);
                s_akk = __ldcg(cand_v + par * G + qw);
                if (q == 0 && (!(v >= lu_tiny<T>() * norm[0]) || norm[0] == T(0))) set_error(err, kDevSingularCoarse);
            }
        }
        __syncthreads();
        const int w = s_w, lw = s_lw;
        for (int m = tid; m < M; m += blockDim.x) {
            if (q + G * m == w) {
                s_pos[m] = k;
                s_done[m] = 1;
            } else if (!s_done[m] && s_pos[m] == k) {
                s_pos[m] = lw;
            }
        }
        const T* prow = slots + (size_t)par * slot_sz + (size_t)s_qw * nd;
        const T akk = s_akk;
        // the pivot row's entries of this thread's columns, loaded before the
        // multipliers so that their latency overlaps the divisions
        T pcs[kRowsCols];
#pragma unroll
        for (int t = 0; t < kRowsCols; ++t) {
            const int c = k + 1 + tid + t * kRowsThreads;
            pcs[t] = c < nd ? __ldcg(prow + c) : T(0);
        }
        __syncthreads();
        for (int m = tid; m < M; m += blockDim.x)
            if (!s_done[m]) {
                const T l = rn_div(rows[(size_t)m * nd + k], akk);
                s_l[m] = l;
                rows[(size_t)m * nd + k] = l;
            }
        __syncthreads();
#pragma unroll
        for (int t = 0; t < kRowsCols; ++t) {
            const int c = k + 1 + tid + t * kRowsThreads;
            if (c < nd)
                for (int m = 0; m < M; ++m)
                    if (!s_done[m]) {
                        T* e = rows + (size_t)m * nd + c;
                        *e = rn_sub(*e, rn_mul(s_l[m], pcs[t]));
                    }
        }
        __syncthreads();
        if (k + 1 < nd) {
            const int np = (k + 1) & 1;
            rows_candidate(nd, k + 1, M, rows, s_pos, s_done, red_v, red_i, cand_v + np * G, cand_i + np * G,
                           cand_p + np * G, slots + (size_t)np * slot_sz);
        }
        if (!grid_barrier(bar, err)) return;
    }
    for (int m = 0; m < M; ++m)
        for (int c = tid; c < nd; c += blockDim.x) a[(size_t)(q + G * m) * nd + c] = rows[(size_t)m * nd + c];
    for (int m = tid; m < M; m += blockDim.x) {
        pos_out[q + G * m] = s_pos[m];
        perm_out[s_pos[m]] = q + G * m;
    }
}

// ---------------------------------------------------------------------------
// Blocked LU (panels of NB columns), same pivots and the same rounded
// operations per entry as the column-by-column paths (the factors are the
// same bits), with three grid barriers per panel instead of one per column:
//  1. one CTA (the last) loads the panel's columns of every active row in
//     logical order into shared memory and factors them column by column
//     (pivot = first largest |value| in logical order, row swaps applied to
//     its copy of the permutation, multipliers, updates of the panel's later
//     columns), then writes the panel back and publishes the permutation;
//  2. all CTAs compute U12, the pivot rows' entries right of the panel, by
//     column slices: each entry minus the panel's earlier columns in order;
//  3. the other CTAs, each holding its cyclically owned rows in shared
//     memory, take the panel's multipliers (and, for pivot rows, U12) and
//     apply the panel's columns in order to their remaining rows right of the
//     panel, then publish those rows for the next panel.
// Every entry thus receives the rounded product and difference of each
// earlier column in column order, as in the column-by-column factorisation.
// ---------------------------------------------------------------------------
template <typename T, int NB>
__global__ void __launch_bounds__(kRowsThreads) lu_panel_kernel(int nd, T* __restrict__ a, const T* __restrict__ norm,
                                                                 int* __restrict__ perm_g, int* __restrict__ pos_g,
                                                                 unsigned* __restrict__ bar, int* err) {
    const int G = gridDim.x, Gr = G - 1, q = blockIdx.x, tid = threadIdx.x;
    const bool panel_cta = q == Gr;
    const int M = panel_cta ? 0 : (nd - q + Gr - 1) / Gr;  // row CTA q owns physical rows q + Gr m
    const int Mmax = (nd + Gr - 1) / Gr;
    extern __shared__ __align__(16) unsigned char lu_panel_sh[];
    T* rows = reinterpret_cast<T*>(lu_panel_sh);                       // row CTAs: [Mmax][nd]
    int* s_pos = reinterpret_cast<int*>(rows + (size_t)Mmax * nd);      // [Mmax] logical positions
    constexpr int PS = NB + 1;  // padded panel row: the threads of a warp hit distinct banks
    T* P = reinterpret_cast<T*>(lu_panel_sh);                          // panel CTA: [nd][PS]
    int* perm_s = reinterpret_cast<int*>(P + (size_t)nd * PS);          // [nd] logical -> physical
    __shared__ T red_v[kRowsThreads / 32];
    __shared__ int red_i[kRowsThreads / 32];
    __shared__ int s_lp;
    __shared__ int s_piv[NB];
    for (int m = 0; m < M; ++m)
        for (int c = tid; c < nd; c += blockDim.x) rows[(size_t)m * nd + c] = __ldcg(a + (size_t)(q + Gr * m) * nd + c);
    for (int m = tid; m < M; m += blockDim.x) s_pos[m] = q + Gr * m;
    for (int r = q * blockDim.x + tid; r < nd; r += G * blockDim.x) {
        perm_g[r] = r;
        pos_g[r] = r;
    }
    if (!grid_barrier(bar, err)) return;
    for (int p0 = 0; p0 < nd; p0 += NB) {
        const int nb = min(NB, nd - p0);
        const int c0 = p0 + nb;
        if (panel_cta) {  // 1. the panel
            const int R = nd - p0;
            for (int l = tid; l < R; l += blockDim.x) perm_s[l] = __ldcg(perm_g + p0 + l);
            __syncthreads();
            for (int e = tid; e < R * nb; e += blockDim.x) {
                const int l = e / nb, c = e - l * nb;
                P[(size_t)l * PS + c] = __ldcg(a + (size_t)perm_s[l] * nd + p0 + c);
            }
            __syncthreads();
            for (int j = 0; j < nb; ++j) {
                T v = T(-1);
                int li = R;
                for (int l = j + tid; l < R; l += blockDim.x) {  // ascending: the first maximum per thread
                    const T av = fabs(P[(size_t)l * PS + j]);
                    if (av > v) {
                        v = av;
                        li = l;
                    }
                }
                cta_argmax(v, li, red_v, red_i);
                if (tid == 0) {
                    s_lp = li;
                    if (!(v >= lu_tiny<T>() * norm[0]) || norm[0] == T(0)) set_error(err, kDevSingularCoarse);
                }
                __syncthreads();
                const int lp = s_lp < R ? s_lp : j;
                if (lp != j) {
                    if (tid < nb) {
                        const T t = P[(size_t)j * PS + tid];
                        P[(size_t)j * PS + tid] = P[(size_t)lp * PS + tid];
                        P[(size_t)lp * PS + tid] = t;
                    }
                    if (tid == 0) {
                        const int t = perm_s[j];
                        perm_s[j] = perm_s[lp];
                        perm_s[lp] = t;
                    }
                }
                __syncthreads();
                const T akk = P[(size_t)j * PS + j];
                for (int l = j + 1 + tid; l < R; l += blockDim.x) {
                    const T lv = rn_div(P[(size_t)l * PS + j], akk);
                    P[(size_t)l * PS + j] = lv;
                    for (int c = j + 1; c < nb; ++c)
                        P[(size_t)l * PS + c] = rn_sub(P[(size_t)l * PS + c], rn_mul(lv, P[(size_t)j * PS + c]));
                }
                __syncthreads();
            }
            for (int e = tid; e < R * nb; e += blockDim.x) {
                const int l = e / nb, c = e - l * nb;
                a[(size_t)perm_s[l] * nd + p0 + c] = P[(size_t)l * PS + c];
            }
            for (int l = tid; l < R; l += blockDim.x) {
                perm_g[p0 + l] = perm_s[l];
                pos_g[perm_s[l]] = p0 + l;
            }
        }
        if (!grid_barrier(bar, err)) return;
        // 2. U12 by column slices over every CTA
        if (tid < nb) s_piv[tid] = __ldcg(perm_g + p0 + tid);
        __syncthreads();
        for (int c = c0 + q * (int)blockDim.x + tid; c < nd; c += G * (int)blockDim.x) {
            T u[NB];
#pragma unroll
            for (int k = 0; k < NB; ++k) {
                if (k < nb) {
                    const T* pr = a + (size_t)s_piv[k] * nd;
                    T x = __ldcg(pr + c);
#pragma unroll
                    for (int j = 0; j < k; ++j) x = rn_sub(x, rn_mul(__ldcg(pr + p0 + j), u[j]));
                    u[k] = x;
                    a[(size_t)s_piv[k] * nd + c] = x;
                }
            }
        }
        if (!grid_barrier(bar, err)) return;
        if (!panel_cta) {  // 3. the owned rows
            for (int m = tid; m < M; m += blockDim.x) s_pos[m] = __ldcg(pos_g + q + Gr * m);
            __syncthreads();
            for (int m = 0; m < M; ++m) {
                const int lp = s_pos[m];
                if (lp < p0) continue;
                const int cend = lp < c0 ? nd : c0;  // pivot rows take U12 as well
                const T* src = a + (size_t)(q + Gr * m) * nd;
                for (int c = p0 + tid; c < cend; c += blockDim.x) rows[(size_t)m * nd + c] = __ldcg(src + c);
            }
            __syncthreads();
            for (int c = c0 + tid; c < nd; c += blockDim.x) {
                T u[NB];
#pragma unroll
                for (int k = 0; k < NB; ++k) u[k] = k < nb ? __ldcg(a + (size_t)s_piv[k] * nd + c) : T(0);
                for (int m = 0; m < M; ++m) {
                    if (s_pos[m] < c0) continue;
                    T* row = rows + (size_t)m * nd;
                    T x = row[c];
#pragma unroll
                    for (int k = 0; k < NB; ++k)
                        if (k < nb) x = rn_sub(x, rn_mul(row[p0 + k], u[k]));
                    row[c] = x;
                    a[(size_t)(q + Gr * m) * nd + c] = x;  // published for the next panel
                }
            }
        }
        if (!grid_barrier(bar, err)) return;
    }
    for (int m = 0; m < M; ++m)
        for (int c = tid; c < nd; c += blockDim.x) a[(size_t)(q + Gr * m) * nd + c] = rows[(size_t)m * nd + c];
}

template <typename T, int NB>
static size_t panel_smem(int nd, int G) {
    const size_t Mmax = (size_t)((nd + G - 2) / (G - 1));
    const size_t row_cta = sizeof(T) * Mmax * nd + sizeof(int) * Mmax;
    const size_t panel_cta = sizeof(T) * (size_t)nd * (NB + 1) + sizeof(int) * (size_t)nd;
    return row_cta > panel_cta ? row_cta : panel_cta;
}

// shared memory of lu_rows_kernel with G CTAs: the owned rows, multipliers,
// logical positions and flags
template <typename T>
static size_t rows_smem(int nd, int G) {
    const size_t M = (size_t)((nd + G - 1) / G);
    return sizeof(T) * (M * nd + M) + 2 * sizeof(int) * M;
}

// shared memory of lu_coop_kernel with G CTAs: perm, pos, the owned-row flags
// (padded to an even count) and multipliers
template <typename T>
static size_t coop_smem(int nd, int G) {
    const int M = (nd + G - 1) / G;
    return sizeof(int) * (2 * (size_t)nd + (size_t)((M + 1) & ~1)) + sizeof(T) * (size_t)M;
}

// scratch of dense_lu_inverse in doubles: multipliers and the norm (nd + 1
// values), two candidate slots (values, rows, logical positions), the
// barrier words, perm and the positions before the copy to piv
long dense_lu_scratch(int nd) { return (long)nd + 1 + 4L * kCoopMaxCtas + 2 + nd + 2; }

// a: the dense matrix (factored in place), inv: its inverse, lt: nd*nd
// scratch (the transposed factors), work: dense_lu_scratch(nd) doubles
template <typename T>
int dense_lu_inverse(int nd, T* a, int* piv, T* inv, T* lt, double* work, int* err, cudaStream_t s) {
    if (nd <= 0) return BAMG_OK;
    int n = 0;
    // carve the scratch by bytes (each piece 8-byte aligned)
    char* w = reinterpret_cast<char*>(work);
    T* col = reinterpret_cast<T*>(w);                     // [nd] multipliers, [1] the norm
    w += 8 * ((size_t)nd + 1);
    T* cand_v = reinterpret_cast<T*>(w);                  // [2 * kCoopMaxCtas]
    w += 8 * (size_t)(2 * kCoopMaxCtas);
    int* cand_i = reinterpret_cast<int*>(w);              // [2 * kCoopMaxCtas]
    w += 8 * (size_t)kCoopMaxCtas;
    unsigned* bar = reinterpret_cast<unsigned*>(w);       // [2]
    w += 8 * 2;
    int* perm = reinterpret_cast<int*>(w);                // [nd]
    int* pos_tmp = perm + nd;                             // [nd]
    w += 4 * (2 * (size_t)nd + 2);
    int* cand_p = reinterpret_cast<int*>(w);              // [2 * kCoopMaxCtas]
    int* pos = piv;  // on return piv holds the logical position of every row
    bool coop_done = false;
    int dev = 0, coop = 0, sms = 0;
    const bool can_coop = cudaGetDevice(&dev) == cudaSuccess &&
                          cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, dev) == cudaSuccess && coop &&
                          cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) == cudaSuccess &&
                          sms <= kCoopMaxCtas;
    if (!can_coop) cudaGetLastError();
    if (nd <= LuSmem<T>::kMax) {
        const size_t smem = sizeof(T) * (size_t)nd * nd;
        BAMG_CUDA_TRY(cudaFuncSetAttribute(lu_smem_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        lu_smem_kernel<T><<<1, kLuThreads, smem, s>>>(nd, a, piv, err);
        n += 1;
    } else {
        BAMG_CUDA_TRY(cudaMemsetAsync(col + nd, 0, sizeof(T), s));
        lu_norm_rows_kernel<T><<<ceil_div((long)nd * 32, 256), 256, 0, s>>>(nd, a, col + nd);
        n += 1;
        int per_sm = 0;
        size_t smem = 0;
        // FP32: blocked, with the owned rows resident in shared memory, when
        // they fit (2048 unknowns: 9.7 ms against 17.8 ms for the per-column
        // kernel below).  FP64 keeps the per-column kernel: there the panel's
        // FP64 work on one SM (nd^2 NB / 2 products and differences, 2 per
        // clock) made the blocked form slower (42.5 against 34.6 ms).
        if constexpr (sizeof(T) == 4) {
            constexpr int NB = 16;  // the panel's nd x (NB + 1) values: 139 KB at nd 2048
            if (can_coop && nd >= 2 * sms && (smem = panel_smem<T, NB>(nd, sms)) > 0 &&
                cudaFuncSetAttribute(lu_panel_kernel<T, NB>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)smem) == cudaSuccess &&
                cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, lu_panel_kernel<T, NB>, kRowsThreads, smem) ==
                    cudaSuccess &&
                per_sm >= 1) {
                BAMG_CUDA_TRY(cudaMemsetAsync(bar, 0, 2 * sizeof(unsigned), s));
                const T* normp = col + nd;
                void* args[] = {&nd, &a, (void*)&normp, &perm, &pos, &bar, &err};
                if (cudaLaunchCooperativeKernel((void*)lu_panel_kernel<T, NB>, dim3(sms), dim3(kRowsThreads), args,
                                                smem, s) == cudaSuccess) {
                    coop_done = true;
                    n += 1;
                } else {
                    (void)cudaGetLastError();  // not launched: the paths below
                }
            } else {
                (void)cudaGetLastError();
            }
        }
        per_sm = 0;
        // rows resident in shared memory when they fit (the candidate rows go
        // through lt, free until the transposition: 2 * sms * nd <= nd^2)
        if (!coop_done && can_coop && nd >= 2 * sms && nd <= kRowsCols * kRowsThreads &&
            (smem = rows_smem<T>(nd, sms)) > 0 &&
            cudaFuncSetAttribute(lu_rows_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) ==
                cudaSuccess &&
            cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, lu_rows_kernel<T>, kRowsThreads, smem) ==
                cudaSuccess &&
            per_sm >= 1) {
            BAMG_CUDA_TRY(cudaMemsetAsync(bar, 0, 2 * sizeof(unsigned), s));
            const T* normp = col + nd;
            T* slots = lt;
            void* args[] = {&nd, &a, (void*)&normp, &cand_v, &cand_i, &cand_p, &slots, &bar, &perm, &pos, &err};
            if (cudaLaunchCooperativeKernel((void*)lu_rows_kernel<T>, dim3(sms), dim3(kRowsThreads), args, smem, s) ==
                cudaSuccess) {
                coop_done = true;
                n += 1;
            } else {
                (void)cudaGetLastError();  // not launched: the paths below
            }
        } else {
            (void)cudaGetLastError();
        }
        per_sm = 0;
        if (!coop_done && can_coop && (smem = coop_smem<T>(nd, sms)) > 0 &&
            cudaFuncSetAttribute(lu_coop_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) ==
                cudaSuccess &&
            cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, lu_coop_kernel<T>, kCoopThreads, smem) ==
                cudaSuccess &&
            per_sm >= 1) {
            BAMG_CUDA_TRY(cudaMemsetAsync(bar, 0, 2 * sizeof(unsigned), s));
            const T* normp = col + nd;
            void* args[] = {&nd, &a, (void*)&normp, &cand_v, &cand_i, &bar, &perm, &pos, &err};
            if (cudaLaunchCooperativeKernel((void*)lu_coop_kernel<T>, dim3(sms), dim3(kCoopThreads), args, smem, s) ==
                cudaSuccess) {
                coop_done = true;
                n += 1;
            } else {
                (void)cudaGetLastError();  // not launched: the per-column path below
            }
        }
        if (!coop_done) {
            for (int k = 0; k < nd; ++k) {
                lu_pivot_kernel<T><<<1, kLuThreads, 0, s>>>(nd, k, a, piv, col, col + nd, err);
                const long m = (long)(nd - k - 1) * (nd - k - 1);
                if (m > 0) {
                    const int blocks = (int)((m + 255) / 256 < 152L * 8 ? (m + 255) / 256 : 152L * 8);
                    lu_update_kernel<T><<<blocks, 256, 0, s>>>(nd, k, a, col);
                    n += 1;
                }
                n += 1;
            }
        }
    }
    if (!coop_done) {  // rows were swapped in place: identity order, positions from the swaps
        swaps_to_pos_kernel<<<ceil_div(nd, 256), 256, 0, s>>>(nd, piv, perm, pos_tmp);
        BAMG_CUDA_TRY(cudaMemcpyAsync(pos, pos_tmp, sizeof(int) * (size_t)nd, cudaMemcpyDeviceToDevice, s));
        n += 1;
    }
    transpose_kernel<T><<<dim3(ceil_div(nd, 32), ceil_div(nd, 32)), dim3(32, 8), 0, s>>>(nd, a, perm, lt);
    constexpr int NC = sizeof(T) == 4 ? 2 : 1;  // (FP64: more columns per CTA measured slower)
    const int groups = (nd + NC - 1) / NC;
    const int cols = groups < 152 * 8 ? groups : 152 * 8;
    lu_inverse_cols_kernel<T, NC><<<cols, kInvThreads, sizeof(T) * (size_t)NC * nd, s>>>(nd, lt, pos, inv);
    return launched(n + 2);
}
template int dense_lu_inverse<double>(int, double*, int*, double*, double*, double*, int*, cudaStream_t);
template int dense_lu_inverse<float>(int, float*, int*, float*, float*, double*, int*, cudaStream_t);

// FP32 copy of a level's values in the field-major layout of vrow (F > 1):
// one warp per block row, entry (k, rr, c) of the block-major FP64 values to
// k0 B^2 + (f len + k - k0) fb B + r B + c with rr = f fb + r, len = k1 - k0
__global__ void convert_fieldmajor_kernel(int n, int b, int fb, const int* __restrict__ rp,
                                          const double* __restrict__ x, float* __restrict__ y) {
    const long i = ((long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (i >= n) return;
    const int k0 = rp[i], k1 = rp[i + 1], len = k1 - k0, bb = b * b;
    for (long e = lane; e < (long)len * bb; e += 32) {
        const int kk = (int)(e / bb), w = (int)(e - (long)kk * bb);
        const int rr = w / b, c = w - rr * b, f = rr / fb, r = rr - f * fb;
        y[(size_t)k0 * bb + ((size_t)f * len + kk) * (fb * b) + (size_t)r * b + c] =
            (float)x[(size_t)(k0 + kk) * bb + w];
    }
}
int launch_convert_fieldmajor(int n, int b, int fb, const int* rp, const double* x, float* y, cudaStream_t s) {
    if (n <= 0) return BAMG_OK;
    convert_fieldmajor_kernel<<<ceil_div((long)n * 32, 256), 256, 0, s>>>(n, b, fb, rp, x, y);
    return launched(1);
}

__global__ void convert_d2f_kernel(long m, const double* __restrict__ x, float* __restrict__ y) {
    for (long e = (long)blockIdx.x * blockDim.x + threadIdx.x; e < m; e += (long)gridDim.x * blockDim.x)
        y[e] = (float)x[e];
}
int launch_convert_d2f(long m, const double* x, float* y, cudaStream_t s) {
    if (m <= 0) return BAMG_OK;
    long g = (m + 255) / 256;
    convert_d2f_kernel<<<(int)(g < 4096 ? g : 4096), 256, 0, s>>>(m, x, y);
    return launched(1);
}

}  // namespace bamg
