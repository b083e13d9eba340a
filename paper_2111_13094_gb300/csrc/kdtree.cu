// kdtree.cu -- the spatial kD-tree of the regions on the GPU (Sec. 4.2
// "Refinement of the spatial kD-tree", Sec. 4.3 "Initialization"):
//
//  k_kd_grid        regular pre-subdivision, heap-numbered nodes
//  k_kd_lookup      leaf of each point by descent
//  binning (k_bin_keys, k_rx_*, k_bin_offsets, k_gather_idx): every sample's
//  leaf, a stable radix sort by leaf, offsets, one gather
//  refinement, as rounds of stable segment partitions:
//    k_kd_tiles     tiles of kKdTile samples, none spanning two segments
//    k_kd_stats     fixed-point position sums of the segments to split
//    k_kd_plan      split plane of each segment (tree node, or mean along the
//                   axis of largest variance)
//    k_kd_count     per tile: samples left of the plane
//    k_kd_scan      which segments split, their new indices, tile prefixes
//    k_kd_scatter   stable partition of every split segment
//    k_kd_segments  new segments, new tree nodes, parents of the new leaves
//  k_kd_gather      the sample streams in the refined order
//  k_gather_state   mixture states copied from the parent regions
//
// Leaves are numbered in tree order (left before right), so a leaf's
// samples are the leaf-th contiguous segment once sorted.  Means and
// variances come from exact integer sums of q = floor(clamp(x, 0, 1) 2^32)
// and q2 = floor(clamp(x, 0, 1)^2 2^32): every implementation places the
// plane identically, and atomics on integers keep the rounds deterministic.
#include "common.cuh"
#include "kernels.h"

namespace sdmm {

constexpr int kKdThreads = 256;               // threads per tile CTA: kKdTile / 256 samples each
constexpr int kKdPer = kKdTile / kKdThreads;
constexpr double kTwo32 = 4294967296.0;

// ---------------------------------------------------------------------------
// Pre-subdivision: every axis split at the centre of its cell, x then y then
// z, `levels` times.  Heap numbering: children of node n are 2n+1 and 2n+2,
// the leaves (depth 3 levels) are the last level, left to right.
__global__ void k_kd_grid(int levels, int32_t* axis, double* split, int32_t* left, int32_t* leaf) {
    const int depth_max = 3 * levels;
    const int64_t n_nodes = (int64_t(1) << (depth_max + 1)) - 1;
    const int64_t n = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (n >= n_nodes) return;
    int d = 0;
    while (((int64_t(1) << (d + 1)) - 1) <= n) ++d;           // depth of node n
    const int64_t p = n - ((int64_t(1) << d) - 1);              // position within its level
    double lo[3] = {0.0, 0.0, 0.0}, hi[3] = {1.0, 1.0, 1.0};
    for (int l = 0; l < d; ++l) {                               // the path from the root
        const int a = l % 3;
        const double mid = 0.5 * (lo[a] + hi[a]);
        if ((p >> (d - 1 - l)) & 1) lo[a] = mid;
        else hi[a] = mid;
    }
    if (d == depth_max) {
        axis[n] = -1;
        split[n] = 0.0;
        left[n] = -1;
        leaf[n] = (int32_t)p;
    } else {
        const int a = d % 3;
        axis[n] = a;
        split[n] = 0.5 * (lo[a] + hi[a]);
        left[n] = (int32_t)(2 * n + 1);
        leaf[n] = -1;
    }
}

__global__ void k_kd_lookup(const int32_t* __restrict__ axis, const double* __restrict__ split,
                            const int32_t* __restrict__ left, const int32_t* __restrict__ leaf, int max_depth,
                            int64_t Q, const float* __restrict__ px, const float* __restrict__ py,
                            const float* __restrict__ pz, int32_t* __restrict__ out) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= Q) return;
    const float x[3] = {px[i], py[i], pz[i]};
    int n = 0;
    for (int d = 0; d <= max_depth && axis[n] >= 0; ++d) {      // bounded by the tree's node count
        const int a = axis[n];
        n = (double)x[a] < split[n] ? left[n] : left[n] + 1;
    }
    out[i] = axis[n] < 0 ? leaf[n] : -1;
}

// ---------------------------------------------------------------------------
// Rounds of segment partitions.  State of a round (workspace, see api.cu):
//   seg_off[S+1] (int64), seg_node[S], seg_parent[S]    the current segments
//   rec[N]                                              (x, y, z, sample index): sample order
// Per segment: flag (split or not), axis, plane, left count; per tile: its
// segment, first sample, left count and its exclusive prefix in the segment.
struct KdRound {
    const int64_t* seg_off;
    const int32_t* seg_node;
    const int64_t* seg_parent;
    int32_t S;
    int32_t* seg_axis;
    double* seg_split;
    float* seg_split_f;          // the smallest float >= seg_split: x < split <=> x < split_f for float x
    int32_t* seg_flag;           // 1: the segment splits this round
    int32_t* seg_new;            // new index of the segment (its left part)
    unsigned long long* seg_sum; // [S][6] fixed-point sums (refinement only)
    unsigned long long* seg_left;
    int32_t* seg_tile0;          // [S+1] first tile of each segment (exclusive prefix of tile counts)
    int32_t* tile_seg;
    int64_t* tile_start;
    int32_t* tile_left;
    int64_t* tile_prefix;
    int32_t* counters;           // [0] tiles, [1] splits
};

// Tiles: ceil(M_s / kKdTile) per segment (empty segments get none), in segment
// order.  One CTA of 1024 threads: the exclusive prefix of the segments' tile
// counts (k_kd_tile_fill then maps tiles to segments in parallel).
__global__ void __launch_bounds__(1024) k_kd_tiles(KdRound k, int64_t max_tiles) {
    __shared__ int64_t s_warp[32];
    __shared__ int64_t s_carry;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    if (tid == 0) s_carry = 0;
    __syncthreads();
    for (int base = 0; base < k.S; base += 1024) {
        const int s = base + tid;
        int64_t nt = 0;
        if (s < k.S) nt = (k.seg_off[s + 1] - k.seg_off[s] + kKdTile - 1) / kKdTile;
        int64_t v = nt;
        for (int d = 1; d < 32; d <<= 1) {
            const int64_t u = __shfl_up_sync(0xffffffffu, v, d);
            if (lane >= d) v += u;
        }
        if (lane == 31) s_warp[warp] = v;
        __syncthreads();
        if (warp == 0) {
            int64_t w = s_warp[lane];
            for (int d = 1; d < 32; d <<= 1) {
                const int64_t u = __shfl_up_sync(0xffffffffu, w, d);
                if (lane >= d) w += u;
            }
            s_warp[lane] = w;
        }
        __syncthreads();
        const int64_t first = s_carry + v - nt + (warp > 0 ? s_warp[warp - 1] : 0);
        if (s < k.S) k.seg_tile0[s] = (int32_t)min(first, max_tiles);
        __syncthreads();
        if (tid == 1023) s_carry = first + nt;
        __syncthreads();
    }
    if (tid == 0) {
        k.seg_tile0[k.S] = (int32_t)min(s_carry, max_tiles);
        k.counters[0] = (int32_t)min(s_carry, max_tiles);
    }
}

// segment and first sample of every tile: the last segment whose first tile
// is <= t (empty segments share their successor's first tile)
__global__ void k_kd_tile_fill(KdRound k) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= k.counters[0]) return;
    int lo = 0, hi = k.S;                        // seg_tile0[lo] <= t < seg_tile0[hi]
    while (hi - lo > 1) {
        const int mid = (lo + hi) >> 1;
        if (k.seg_tile0[mid] <= t) lo = mid;
        else hi = mid;
    }
    k.tile_seg[t] = lo;
    k.tile_start[t] = k.seg_off[lo] + (int64_t)(t - k.seg_tile0[lo]) * kKdTile;
}

// q = floor(clamp(x, 0, 1) 2^32) and q2 = floor(clamp(x, 0, 1)^2 2^32), exactly,
// from the float's integer mantissa and exponent (x = m 2^e), in integer
// arithmetic (the FP64 units of this GPU are few)
__device__ __forceinline__ void fixed_point(float x, unsigned long long& q, unsigned long long& q2) {
    if (!(x > 0.f)) {                                     // also NaN
        q = q2 = 0ull;
        return;
    }
    if (x >= 1.f) {
        q = q2 = 4294967296ull;
        return;
    }
    const uint32_t b = __float_as_uint(x);
    const int ef = (int)(b >> 23);                        // biased exponent, 0 for subnormals
    const unsigned long long m = ef ? ((b & 0x7FFFFFu) | 0x800000u) : (b & 0x7FFFFFu);
    const int e = (ef ? ef : 1) - 150;                   // x = m 2^e, e <= -24 here
    const int s1 = e + 32, s2 = 2 * e + 32;
    q = s1 >= 0 ? (m << s1) : (-s1 >= 64 ? 0ull : (m >> -s1));
    const unsigned long long mm = m * m;                 // < 2^48
    q2 = s2 >= 0 ? (mm << s2) : (-s2 >= 64 ? 0ull : (mm >> -s2));
}

// fixed-point sums of the samples of segments holding more than c of them
__global__ void __launch_bounds__(kKdThreads) k_kd_stats(KdRound k, const float4* __restrict__ rec, int64_t c) {
    __shared__ unsigned long long s_red[kKdThreads / 32][6];
    const int t = blockIdx.x;
    if (t >= k.counters[0]) return;
    const int s = k.tile_seg[t];
    const int64_t end = k.seg_off[s + 1];
    const int64_t M = end - k.seg_off[s];
    if (M <= c) return;                                        // (uniform per CTA)
    const int64_t i0 = k.tile_start[t] + threadIdx.x;
    unsigned long long v[6] = {0ull, 0ull, 0ull, 0ull, 0ull, 0ull};
#pragma unroll
    for (int q = 0; q < kKdPer; ++q) {
        const int64_t i = i0 + q * kKdThreads;
        if (i < end) {
            const float4 p = rec[i];
            unsigned long long a, b;
            fixed_point(p.x, a, b);
            v[0] += a, v[3] += b;
            fixed_point(p.y, a, b);
            v[1] += a, v[4] += b;
            fixed_point(p.z, a, b);
            v[2] += a, v[5] += b;
        }
    }
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int q = 0; q < 6; ++q) {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v[q] += __shfl_xor_sync(0xffffffffu, v[q], o);
        if (lane == 0) s_red[warp][q] = v[q];
    }
    __syncthreads();
    if (threadIdx.x < 6) {
        unsigned long long a = 0ull;
        for (int w = 0; w < kKdThreads / 32; ++w) a += s_red[w][threadIdx.x];
        atomicAdd(k.seg_sum + (int64_t)s * 6 + threadIdx.x, a);
    }
}

// Split plane of every segment holding more than c samples: the mean along
// the axis of largest variance (lowest axis on ties), from the sums.
__global__ void k_kd_plan(KdRound k, int64_t c) {
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= k.S) return;
    const int64_t M = k.seg_off[s + 1] - k.seg_off[s];
    int a = -1;
    double pl = 0.0;
    if (M > c) {
        double best = -1.0;
        for (int q = 0; q < 3; ++q) {
            const double S1 = (double)k.seg_sum[(int64_t)s * 6 + q];
            const double S2 = (double)k.seg_sum[(int64_t)s * 6 + 3 + q];
            const double mean = __ddiv_rn(__ddiv_rn(S1, (double)M), kTwo32);
            const double var = __dsub_rn(__ddiv_rn(__ddiv_rn(S2, (double)M), kTwo32), __dmul_rn(mean, mean));
            if (var > best) {
                best = var;
                a = q;
                pl = mean;
            }
        }
    }
    k.seg_axis[s] = a;
    k.seg_split[s] = pl;
    k.seg_split_f[s] = __double2float_ru(pl);
    k.seg_left[s] = 0ull;
}

// per tile: samples strictly left of the plane (x[axis] < split)
__global__ void __launch_bounds__(kKdThreads) k_kd_count(KdRound k, const float4* __restrict__ rec) {
    __shared__ int s_red[kKdThreads / 32];
    const int t = blockIdx.x;
    if (t >= k.counters[0]) return;
    const int s = k.tile_seg[t];
    const int a = k.seg_axis[s];
    const int64_t end = k.seg_off[s + 1];
    const float pl = k.seg_split_f[s];
    const int64_t i0 = k.tile_start[t] + threadIdx.x;
    int f = 0;
#pragma unroll
    for (int q = 0; q < kKdPer; ++q) {
        const int64_t i = i0 + q * kKdThreads;
        if (a >= 0 && i < end) {
            const float4 p = rec[i];
            const float x = a == 0 ? p.x : (a == 1 ? p.y : p.z);
            f += x < pl ? 1 : 0;
        }
    }
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    int n = f;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) n += __shfl_xor_sync(0xffffffffu, n, o);
    if (lane == 0) s_red[warp] = n;
    __syncthreads();
    if (threadIdx.x == 0) {
        int tot = 0;
        for (int w = 0; w < kKdThreads / 32; ++w) tot += s_red[w];
        k.tile_left[t] = tot;
        if (a >= 0) atomicAdd(k.seg_left + s, (unsigned long long)tot);
    }
}

// Which segments split (both sides non-empty), their new indices, and the
// exclusive prefix of each tile's left count within its segment.  One CTA of
// 1024 threads.
__global__ void __launch_bounds__(1024) k_kd_scan(KdRound k) {
    __shared__ int32_t s_warp[32];
    __shared__ int32_t s_carry;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    if (tid == 0) s_carry = 0;
    __syncthreads();
    for (int base = 0; base < k.S; base += 1024) {
        const int s = base + tid;
        int f = 0;
        if (s < k.S && k.seg_axis[s] >= 0) {
            const int64_t M = k.seg_off[s + 1] - k.seg_off[s];
            const int64_t L = (int64_t)k.seg_left[s];
            f = (L > 0 && L < M) ? 1 : 0;
        }
        int v = f;
        for (int d = 1; d < 32; d <<= 1) {
            const int u = __shfl_up_sync(0xffffffffu, v, d);
            if (lane >= d) v += u;
        }
        if (lane == 31) s_warp[warp] = v;
        __syncthreads();
        if (warp == 0) {
            int w = s_warp[lane];
            for (int d = 1; d < 32; d <<= 1) {
                const int u = __shfl_up_sync(0xffffffffu, w, d);
                if (lane >= d) w += u;
            }
            s_warp[lane] = w;
        }
        __syncthreads();
        const int before = s_carry + v - f + (warp > 0 ? s_warp[warp - 1] : 0);
        if (s < k.S) {
            k.seg_flag[s] = f;
            k.seg_new[s] = s + before;
        }
        __syncthreads();
        if (tid == 1023) s_carry = before + f;
        __syncthreads();
    }
    if (tid == 0) k.counters[1] = s_carry;
    __syncthreads();
    // tile prefixes (tiles of a segment are consecutive)
    const int nt = k.counters[0];
    __shared__ int64_t s_run;
    __shared__ int64_t s_w64[32];
    if (tid == 0) s_run = 0;
    __syncthreads();
    for (int base = 0; base < nt; base += 1024) {
        const int t = base + tid;
        int64_t c = t < nt ? k.tile_left[t] : 0;
        int64_t v = c;
        for (int d = 1; d < 32; d <<= 1) {
            const int64_t u = __shfl_up_sync(0xffffffffu, v, d);
            if (lane >= d) v += u;
        }
        if (lane == 31) s_w64[warp] = v;
        __syncthreads();
        if (warp == 0) {
            int64_t w = s_w64[lane];
            for (int d = 1; d < 32; d <<= 1) {
                const int64_t u = __shfl_up_sync(0xffffffffu, w, d);
                if (lane >= d) w += u;
            }
            s_w64[lane] = w;
        }
        __syncthreads();
        const int64_t excl = s_run + v - c + (warp > 0 ? s_w64[warp - 1] : 0);
        if (t < nt) k.tile_prefix[t] = excl;          // global exclusive prefix
        __syncthreads();
        if (tid == 1023) s_run = excl + c;
        __syncthreads();
    }
}

// Stable partition: within a split segment, left samples first (in order),
// then the right ones (in order); other segments are copied.  Thread j of the
// CTA holds samples j, j + 256, j + 512, j + 768 of the tile.
__global__ void __launch_bounds__(kKdThreads) k_kd_scatter(KdRound k, const float4* __restrict__ rec_in,
                                                         float4* __restrict__ rec_out) {
    constexpr int W = kKdThreads / 32;
    __shared__ int s_cnt[kKdPer][W];
    const int t = blockIdx.x;
    if (t >= k.counters[0]) return;
    const int s = k.tile_seg[t];
    const int64_t o0 = k.seg_off[s], o1 = k.seg_off[s + 1];
    const int64_t i0 = k.tile_start[t] + threadIdx.x;
    float4 p[kKdPer];
#pragma unroll
    for (int q = 0; q < kKdPer; ++q) {
        const int64_t i = i0 + q * kKdThreads;
        p[q] = i < o1 ? rec_in[i] : make_float4(0.f, 0.f, 0.f, 0.f);
    }
    if (!k.seg_flag[s]) {
#pragma unroll
        for (int q = 0; q < kKdPer; ++q)
            if (i0 + q * kKdThreads < o1) rec_out[i0 + q * kKdThreads] = p[q];
        return;                                               // (uniform per CTA)
    }
    const int a = k.seg_axis[s];
    const float pl = k.seg_split_f[s];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    int f[kKdPer], rank_w[kKdPer];
#pragma unroll
    for (int q = 0; q < kKdPer; ++q) {
        const bool in = i0 + q * kKdThreads < o1;
        const float x = a == 0 ? p[q].x : (a == 1 ? p[q].y : p[q].z);
        f[q] = (in && x < pl) ? 1 : 0;
        const unsigned bal = __ballot_sync(0xffffffffu, f[q]);
        rank_w[q] = __popc(bal & ((1u << lane) - 1u));
        if (lane == 0) s_cnt[q][warp] = __popc(bal);
    }
    __syncthreads();
    const int64_t lpre = k.tile_prefix[t] - k.tile_prefix[k.seg_tile0[s]];   // left samples of earlier tiles
    const int64_t L = (int64_t)k.seg_left[s];
    int before = 0;                                // left samples of the tile before (q, warp)
#pragma unroll
    for (int q = 0; q < kKdPer; ++q) {
        int wb = 0;
        for (int w = 0; w < W; ++w) wb += w < warp ? s_cnt[q][w] : 0;
        const int64_t i = i0 + q * kKdThreads;
        if (i < o1) {
            const int lrank = before + wb + rank_w[q];
            const int64_t pos_in_seg = i - o0;
            const int64_t dst = f[q] ? o0 + lpre + lrank : o0 + L + (pos_in_seg - (lpre + lrank));
            rec_out[dst] = p[q];
        }
        for (int w = 0; w < W; ++w) before += s_cnt[q][w];
    }
}

// New segments and the tree: two new leaf nodes per split, appended from node
// n_nodes on, and leaf indices of kept leaves.
__global__ void k_kd_segments(KdRound k, int32_t* tree_axis, double* tree_split, int32_t* tree_left,
                              int32_t* tree_leaf, int32_t n_nodes, int64_t* seg_off_out, int32_t* seg_node_out,
                              int64_t* seg_parent_out, int64_t N) {
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= k.S) return;
    const int ns = k.seg_new[s];
    const int32_t node = k.seg_node[s];
    const int64_t off = k.seg_off[s];
    const int64_t par = k.seg_parent[s];
    if (k.seg_flag[s]) {
        const int64_t L = (int64_t)k.seg_left[s];
        const int32_t l = n_nodes + 2 * (ns - s);
        tree_axis[node] = k.seg_axis[s];
        tree_split[node] = k.seg_split[s];
        tree_left[node] = l;
        tree_leaf[node] = -1;
        tree_axis[l] = -1;
        tree_axis[l + 1] = -1;
        tree_split[l] = tree_split[l + 1] = 0.0;
        tree_left[l] = tree_left[l + 1] = -1;
        tree_leaf[l] = ns;
        tree_leaf[l + 1] = ns + 1;
        seg_node_out[ns] = l;
        seg_node_out[ns + 1] = l + 1;
        seg_off_out[ns] = off;
        seg_off_out[ns + 1] = off + L;
        seg_parent_out[ns] = par;
        seg_parent_out[ns + 1] = par;
    } else {
        tree_leaf[node] = ns;
        seg_node_out[ns] = node;
        seg_off_out[ns] = off;
        seg_parent_out[ns] = par;
    }
    if (s == k.S - 1) seg_off_out[ns + 1 + k.seg_flag[s]] = N;
}

// leaf -> node of every leaf node (initial segments of a refinement)
__global__ void k_kd_leaf_nodes(const int32_t* __restrict__ axis, const int32_t* __restrict__ leaf, int32_t n_nodes,
                                int32_t* seg_node) {
    const int n = blockIdx.x * blockDim.x + threadIdx.x;
    if (n < n_nodes && axis[n] < 0) seg_node[leaf[n]] = n;
}

// records (x, y, z, i): the positions travel with the sample index, so every
// round reads them in order
__global__ void k_kd_init(float4* rec, int64_t N, const float* __restrict__ px, const float* __restrict__ py,
                          const float* __restrict__ pz, int64_t* parent, int32_t S) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < N) rec[i] = make_float4(px[i], py[i], pz[i], __int_as_float((int32_t)i));
    if (parent != nullptr && i < S) parent[i] = i;
}

__global__ void k_kd_gather(int64_t N, const float4* __restrict__ rec, BatchDesc in, BatchDesc out) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N) return;
    const int32_t j = __float_as_int(rec[i].w);
#pragma unroll
    for (int q = 0; q < 7; ++q) const_cast<float*>(out.p[q])[i] = in.p[q][j];
}

// Mixture states of new regions copied from their source regions (the
// parent leaf's mixture is copied into both children, Sec. 4.2).
__global__ void k_gather_state(int K, int64_t R_out, const int64_t* __restrict__ src, sdmm_state in,
                               sdmm_state out) {
    const int64_t r = blockIdx.x;
    if (r >= R_out) return;
    const int64_t q = src[r];
    for (int e = threadIdx.x; e < K; e += blockDim.x) {
        const int64_t a = r * K + e, b = q * K + e;
        out.pi[a] = in.pi[b];
        out.S0[a] = in.S0[b];
        for (int c = 0; c < 3; ++c) {
            out.mu_x[a * 3 + c] = in.mu_x[b * 3 + c];
            out.mu_w[a * 3 + c] = in.mu_w[b * 3 + c];
        }
        for (int p = 0; p < 15; ++p) {
            out.L[a * 15 + p] = in.L[b * 15 + p];
            out.S2[a * 15 + p] = in.S2[b * 15 + p];
        }
        for (int p = 0; p < kE; ++p) out.etab[a * kE + p] = in.etab[b * kE + p];
        for (int p = 0; p < kQ; ++p) out.qtab[a * kQ + p] = in.qtab[b * kQ + p];
    }
    if (threadIdx.x == 0) {
        out.Wbar[r] = in.Wbar[q];
        out.n_seen[r] = in.n_seen[q];
        out.step_j[r] = in.step_j[q];
        out.status[r] = in.status[q];
    }
}

// ---------------------------------------------------------------------------
cudaError_t launch_kd_grid(cudaStream_t s, int levels, int32_t* axis, double* split, int32_t* left,
                           int32_t* leaf) {
    const int64_t n = (int64_t(1) << (3 * levels + 1)) - 1;
    k_kd_grid<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(levels, axis, split, left, leaf);
    return cudaGetLastError();
}

cudaError_t launch_kd_lookup(cudaStream_t s, const int32_t* axis, const double* split, const int32_t* left,
                             const int32_t* leaf, int max_depth, int64_t Q, const float* px, const float* py,
                             const float* pz, int32_t* out) {
    if (Q == 0) return cudaSuccess;
    k_kd_lookup<<<(unsigned)((Q + 255) / 256), 256, 0, s>>>(axis, split, left, leaf, max_depth, Q, px, py, pz,
                                                           out);
    return cudaGetLastError();
}

cudaError_t launch_gather_state(cudaStream_t s, int K, int64_t R_out, const int64_t* src, const sdmm_state& in,
                                const sdmm_state& out) {
    if (R_out == 0) return cudaSuccess;
    k_gather_state<<<(unsigned)R_out, 32, 0, s>>>(K, R_out, src, in, out);
    return cudaGetLastError();
}

// One refinement over all rounds (host loop; one 4-byte read-back per round).
// ws layout in KdWork (api.cu).
cudaError_t kd_rounds(cudaStream_t st, const KdWork& w, int64_t c, int32_t* tree_axis,
                      double* tree_split, int32_t* tree_left, int32_t* tree_leaf, int32_t* n_nodes,
                      int32_t* n_leaves, int32_t cap_nodes, int32_t cap_leaves, int32_t S0, int64_t N,
                      const float4** rec_final,
                      int64_t** seg_off_final, int64_t** seg_parent_final, int32_t* S_final, int* overflow) {
    int32_t S = S0;
    int cur = 0;
    *overflow = 0;
    for (int round = 0; round < 64; ++round) {
        KdRound k{};
        k.seg_off = w.seg_off[cur];
        k.seg_node = w.seg_node[cur];
        k.seg_parent = w.seg_parent[cur];
        k.S = S;
        k.seg_axis = w.seg_axis;
        k.seg_split = w.seg_split;
        k.seg_split_f = w.seg_split_f;
        k.seg_flag = w.seg_flag;
        k.seg_new = w.seg_new;
        k.seg_sum = w.seg_sum;
        k.seg_left = w.seg_left;
        k.seg_tile0 = w.seg_tile0;
        k.tile_seg = w.tile_seg;
        k.tile_start = w.tile_start;
        k.tile_left = w.tile_left;
        k.tile_prefix = w.tile_prefix;
        k.counters = w.counters;
        const int64_t max_tiles = w.max_tiles;
        cudaError_t e;
        k_kd_tiles<<<1, 1024, 0, st>>>(k, max_tiles);
        k_kd_tile_fill<<<(unsigned)((max_tiles + 255) / 256), 256, 0, st>>>(k);
        if ((e = cudaMemsetAsync(w.seg_sum, 0, sizeof(unsigned long long) * 6 * (size_t)S, st)) != cudaSuccess)
            return e;
        k_kd_stats<<<(unsigned)max_tiles, kKdThreads, 0, st>>>(k, w.rec[cur & 1], c);
        k_kd_plan<<<(S + 255) / 256, 256, 0, st>>>(k, c);
        k_kd_count<<<(unsigned)max_tiles, kKdThreads, 0, st>>>(k, w.rec[cur & 1]);
        k_kd_scan<<<1, 1024, 0, st>>>(k);
        int32_t splits = 0;
        if ((e = cudaMemcpyAsync(&splits, w.counters + 1, sizeof(int32_t), cudaMemcpyDeviceToHost, st)) != cudaSuccess)
            return e;
        if ((e = cudaStreamSynchronize(st)) != cudaSuccess) return e;
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
        if (splits == 0) break;
        if (S + splits > cap_leaves || *n_nodes + 2 * splits > cap_nodes) {
            *overflow = 1;
            return cudaSuccess;
        }
        k_kd_scatter<<<(unsigned)max_tiles, kKdThreads, 0, st>>>(k, w.rec[cur & 1], w.rec[(cur + 1) & 1]);
        k_kd_segments<<<(S + 255) / 256, 256, 0, st>>>(k, tree_axis, tree_split, tree_left, tree_leaf,
                                                      *n_nodes, w.seg_off[cur ^ 1], w.seg_node[cur ^ 1],
                                                      w.seg_parent[cur ^ 1], N);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
        *n_nodes += 2 * splits;
        *n_leaves += splits;
        S += splits;
        cur ^= 1;
    }
    *rec_final = w.rec[cur & 1];
    *seg_off_final = w.seg_off[cur];
    *seg_parent_final = w.seg_parent[cur];
    *S_final = S;
    return cudaSuccess;
}

cudaError_t launch_kd_prepare(cudaStream_t st, const KdWork& w, const int32_t* tree_axis,
                              const int32_t* tree_leaf, int32_t n_nodes, int32_t S0, const int64_t* offsets_in,
                              int64_t N, const float* px, const float* py, const float* pz) {
    k_kd_init<<<(unsigned)((std::max<int64_t>(N, S0) + 255) / 256), 256, 0, st>>>(w.rec[0], N, px, py, pz,
                                                                                 w.seg_parent[0], S0);
    cudaError_t e = cudaMemcpyAsync(w.seg_off[0], offsets_in, sizeof(int64_t) * (S0 + 1), cudaMemcpyDeviceToDevice, st);
    if (e != cudaSuccess) return e;
    k_kd_leaf_nodes<<<(n_nodes + 255) / 256, 256, 0, st>>>(tree_axis, tree_leaf, n_nodes, w.seg_node[0]);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Binning into a fixed tree (Sec. 4.2: the samples of a round go to the leaf
// that contains them): every sample's leaf by descent, then a stable LSD
// radix sort of (leaf, index) pairs with 8-bit digits, the leaf offsets from
// the sorted keys, and one gather of the seven streams.  Stability keeps the
// samples of a leaf in their input order.
constexpr int kRxThreads = 256, kRxPer = 8, kRxTile = kRxThreads * kRxPer;   // keys per tile
constexpr int kRxScan = 4096;                                                 // entries per scan block

// the float threshold of every node: the smallest float >= split (exact test)
__global__ void k_kd_split_f(const double* __restrict__ split, int32_t n_nodes, float* __restrict__ split_f) {
    const int n = blockIdx.x * blockDim.x + threadIdx.x;
    if (n < n_nodes) split_f[n] = __double2float_ru(split[n]);
}

__global__ void k_bin_keys(const int32_t* __restrict__ axis, const float* __restrict__ split,
                           const int32_t* __restrict__ left, const int32_t* __restrict__ leaf, int max_depth,
                           int64_t N, const float* __restrict__ px, const float* __restrict__ py,
                           const float* __restrict__ pz, uint32_t* __restrict__ key, uint32_t* __restrict__ idx) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N) return;
    const float x[3] = {px[i], py[i], pz[i]};
    int n = 0;
    for (int d = 0; d <= max_depth && axis[n] >= 0; ++d) {      // bounded by the tree's node count
        const int a = axis[n];
        n = x[a] < split[n] ? left[n] : left[n] + 1;
    }
    key[i] = axis[n] < 0 ? (uint32_t)leaf[n] : 0u;
    idx[i] = (uint32_t)i;
}

// per tile of 2048 keys: counts of each digit, digit-major (hist[d T + tile])
__global__ void __launch_bounds__(kRxThreads) k_rx_hist(const uint32_t* __restrict__ key, int64_t N, int shift,
                                                      int T, uint32_t* __restrict__ hist) {
    __shared__ uint32_t h[256];
    h[threadIdx.x] = 0u;
    __syncthreads();
    const int64_t base = (int64_t)blockIdx.x * kRxTile;
#pragma unroll
    for (int q = 0; q < kRxPer; ++q) {
        const int64_t i = base + q * kRxThreads + threadIdx.x;
        if (i < N) atomicAdd(&h[(key[i] >> shift) & 255u], 1u);
    }
    __syncthreads();
    hist[(int64_t)threadIdx.x * T + blockIdx.x] = h[threadIdx.x];
}

// exclusive scan of M counts in place: block sums, a one-CTA scan of the
// sums, then each block's own scan plus its offset
__global__ void __launch_bounds__(1024) k_rx_scan_sums(const uint32_t* __restrict__ a, int64_t M,
                                                     uint32_t* __restrict__ bsum) {
    __shared__ uint32_t s[32];
    const int64_t b0 = (int64_t)blockIdx.x * kRxScan;
    uint32_t v = 0u;
#pragma unroll
    for (int q = 0; q < kRxScan / 1024; ++q) {
        const int64_t i = b0 + q * 1024 + threadIdx.x;
        if (i < M) v += a[i];
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if ((threadIdx.x & 31) == 0) s[threadIdx.x >> 5] = v;
    __syncthreads();
    if (threadIdx.x < 32) {
        uint32_t w = s[threadIdx.x];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) w += __shfl_xor_sync(0xffffffffu, w, o);
        if (threadIdx.x == 0) bsum[blockIdx.x] = w;
    }
}

__device__ __forceinline__ uint32_t block_exclusive_1024(uint32_t v, uint32_t* s_warp, uint32_t* total) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    uint32_t x = v;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
        const uint32_t u = __shfl_up_sync(0xffffffffu, x, d);
        if (lane >= d) x += u;
    }
    if (lane == 31) s_warp[warp] = x;
    __syncthreads();
    if (warp == 0) {
        uint32_t w = s_warp[lane];
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
            const uint32_t u = __shfl_up_sync(0xffffffffu, w, d);
            if (lane >= d) w += u;
        }
        s_warp[lane] = w;
    }
    __syncthreads();
    const uint32_t ex = x - v + (warp > 0 ? s_warp[warp - 1] : 0u);
    *total = s_warp[31];
    __syncthreads();
    return ex;
}

__global__ void __launch_bounds__(1024) k_rx_scan_top(uint32_t* __restrict__ bsum, int nb) {
    __shared__ uint32_t s_warp[32];
    uint32_t carry = 0u;
    for (int base = 0; base < nb; base += 1024) {
        const int i = base + threadIdx.x;
        const uint32_t v = i < nb ? bsum[i] : 0u;
        uint32_t tot;
        const uint32_t ex = block_exclusive_1024(v, s_warp, &tot);
        if (i < nb) bsum[i] = carry + ex;
        carry += tot;
    }
}

__global__ void __launch_bounds__(1024) k_rx_scan_down(uint32_t* __restrict__ a, int64_t M,
                                                     const uint32_t* __restrict__ bsum) {
    __shared__ uint32_t s_warp[32];
    const int64_t b0 = (int64_t)blockIdx.x * kRxScan;
    uint32_t carry = bsum[blockIdx.x];
    for (int q = 0; q < kRxScan / 1024; ++q) {
        const int64_t i = b0 + q * 1024 + threadIdx.x;
        const uint32_t v = i < M ? a[i] : 0u;
        uint32_t tot;
        const uint32_t ex = block_exclusive_1024(v, s_warp, &tot);
        if (i < M) a[i] = carry + ex;
        carry += tot;
    }
}

// stable scatter of one digit: the tile's keys in eight ordered sub-rounds of
// 256; within a sub-round, rank among equal digits by warp, then lane
__global__ void __launch_bounds__(kRxThreads) k_rx_scatter(const uint32_t* __restrict__ key_in,
                                                         const uint32_t* __restrict__ idx_in,
                                                         uint32_t* __restrict__ key_out,
                                                         uint32_t* __restrict__ idx_out, int64_t N, int shift,
                                                         int T, const uint32_t* __restrict__ off) {
    constexpr int W = kRxThreads / 32;
    __shared__ uint32_t s_carry[256];
    __shared__ uint32_t s_wc[W][256];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int tile = blockIdx.x;
    s_carry[tid] = off[(int64_t)tid * T + tile];
    const int64_t base = (int64_t)tile * kRxTile;
    for (int r = 0; r < kRxPer; ++r) {
#pragma unroll
        for (int w = 0; w < W; ++w) s_wc[w][tid] = 0u;
        __syncthreads();
        const int64_t i = base + r * kRxThreads + tid;
        const bool valid = i < N;
        const uint32_t k = valid ? key_in[i] : 0u;
        const uint32_t v = valid ? idx_in[i] : 0u;
        const uint32_t d = valid ? (k >> shift) & 255u : 256u;   // invalid lanes only match each other
        const unsigned peers = __match_any_sync(0xffffffffu, d);
        const int rank = __popc(peers & ((1u << lane) - 1u));
        if (valid && rank == 0) s_wc[warp][d] = (uint32_t)__popc(peers);
        __syncthreads();
        if (valid) {
            uint32_t pre = 0u;
            for (int w = 0; w < warp; ++w) pre += s_wc[w][d];
            const uint32_t dst = s_carry[d] + pre + (uint32_t)rank;
            key_out[dst] = k;
            idx_out[dst] = v;
        }
        __syncthreads();
        uint32_t add = 0u;
#pragma unroll
        for (int w = 0; w < W; ++w) add += s_wc[w][tid];
        s_carry[tid] += add;
        __syncthreads();
    }
}

// offsets[l] = first position of leaf l in the sorted keys (S + 1 entries)
__global__ void k_bin_offsets(const uint32_t* __restrict__ key, int64_t N, int32_t S, int64_t* __restrict__ offsets) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i > N) return;
    const int64_t prev = i > 0 ? (int64_t)key[i - 1] : -1;
    const int64_t cur = i < N ? (int64_t)key[i] : (int64_t)S;
    for (int64_t l = prev + 1; l <= cur; ++l) offsets[l] = i;
}

__global__ void k_gather_idx(int64_t N, const uint32_t* __restrict__ idx, BatchDesc in, BatchDesc out) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N) return;
    const uint32_t j = idx[i];
#pragma unroll
    for (int q = 0; q < 7; ++q) const_cast<float*>(out.p[q])[i] = in.p[q][j];
}

// One counting pass for trees of at most 1024 leaves (10-bit keys): tiles of
// 8192 keys, so the digit counts take as much room as the 8-bit passes'
// (1024 x N / 8192 = 256 x N / 2048), and the scatter moves the seven sample
// streams themselves (read in order, written to their leaf's run) instead of
// an index that a gather would follow at random afterwards.
constexpr int kCsBits = 10, kCsDigits = 1 << kCsBits, kCsPer = 32, kCsTile = kRxThreads * kCsPer;

__global__ void __launch_bounds__(kRxThreads) k_cs_hist(const uint32_t* __restrict__ key, int64_t N, int T,
                                                      uint32_t* __restrict__ hist) {
    __shared__ uint32_t h[kCsDigits];
    for (int d = threadIdx.x; d < kCsDigits; d += kRxThreads) h[d] = 0u;
    __syncthreads();
    const int64_t base = (int64_t)blockIdx.x * kCsTile;
    for (int q = 0; q < kCsPer; ++q) {
        const int64_t i = base + q * kRxThreads + threadIdx.x;
        if (i < N) atomicAdd(&h[key[i] & (kCsDigits - 1)], 1u);
    }
    __syncthreads();
    for (int d = threadIdx.x; d < kCsDigits; d += kRxThreads) hist[(int64_t)d * T + blockIdx.x] = h[d];
}

// stable scatter of the keys and the seven streams: the tile's keys in 32
// ordered sub-rounds of 256; within a sub-round, rank among equal keys by
// warp, then lane (warp counts kept only for the keys present)
__global__ void __launch_bounds__(kRxThreads) k_cs_scatter(const uint32_t* __restrict__ key_in,
                                                         uint32_t* __restrict__ key_out, int64_t N, int T,
                                                         const uint32_t* __restrict__ off, BatchDesc in,
                                                         BatchDesc out) {
    constexpr int W = kRxThreads / 32;
    __shared__ uint32_t s_carry[kCsDigits];
    __shared__ uint32_t s_wc[W][kCsDigits];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int tile = blockIdx.x;
    for (int d = tid; d < kCsDigits; d += kRxThreads) {
        s_carry[d] = off[(int64_t)d * T + tile];
#pragma unroll
        for (int w = 0; w < W; ++w) s_wc[w][d] = 0u;
    }
    __syncthreads();
    const int64_t base = (int64_t)tile * kCsTile;
    for (int r = 0; r < kCsPer; ++r) {
        const int64_t i = base + r * kRxThreads + tid;
        const bool valid = i < N;
        const uint32_t k = valid ? key_in[i] : 0u;
        const uint32_t d = valid ? (k & (kCsDigits - 1)) : (uint32_t)kCsDigits;   // invalid lanes match only each other
        const unsigned peers = __match_any_sync(0xffffffffu, d);
        const int rank = __popc(peers & ((1u << lane) - 1u));
        const bool lead = valid && rank == 0;
        if (lead) s_wc[warp][d] = (uint32_t)__popc(peers);
        __syncthreads();
        if (valid) {
            uint32_t pre = 0u;
            for (int w = 0; w < warp; ++w) pre += s_wc[w][d];
            const uint32_t dst = s_carry[d] + pre + (uint32_t)rank;
            key_out[dst] = k;
#pragma unroll
            for (int q = 0; q < 7; ++q) const_cast<float*>(out.p[q])[dst] = in.p[q][i];
        }
        __syncthreads();
        if (lead) {
            atomicAdd(&s_carry[d], (uint32_t)__popc(peers));
            s_wc[warp][d] = 0u;
        }
        __syncthreads();
    }
}

int64_t rx_tiles(int64_t N) { return (N + kRxTile - 1) / kRxTile; }
// digit-count entries of the larger of the two schemes (8-bit passes; the
// one 10-bit pass, whose tile count rounds up separately)
int64_t rx_hist_entries(int64_t N) {
    return std::max<int64_t>(256 * rx_tiles(N), (int64_t)kCsDigits * ((N + kCsTile - 1) / kCsTile));
}
int64_t rx_scan_blocks(int64_t N) { return (rx_hist_entries(N) + kRxScan - 1) / kRxScan; }

cudaError_t launch_kd_bin(cudaStream_t st, const KdWork& w, const int32_t* axis, const double* split,
                          const int32_t* left, const int32_t* leaf, int32_t n_nodes, int32_t n_leaves, int64_t N,
                          const float* px, const float* py, const float* pz, const BatchDesc& in,
                          const BatchDesc& out, int64_t* offsets) {
    uint32_t* key[2] = {reinterpret_cast<uint32_t*>(w.rec[0]), reinterpret_cast<uint32_t*>(w.rec[1])};
    uint32_t* idx[2] = {key[0] + N, key[1] + N};
    if (N > 0) {
        k_kd_split_f<<<(n_nodes + 255) / 256, 256, 0, st>>>(split, n_nodes, w.split_f);
        k_bin_keys<<<(unsigned)((N + 255) / 256), 256, 0, st>>>(axis, w.split_f, left, leaf, n_nodes, N, px, py,
                                                               pz, key[0], idx[0]);
        int bits = 0;
        while (bits < 32 && (int64_t(1) << bits) < (int64_t)n_leaves) ++bits;
        if (bits <= kCsBits) {                    // one counting pass moving the streams
            const int T = (int)((N + kCsTile - 1) / kCsTile);
            const int64_t M = (int64_t)kCsDigits * T;
            const int nb = (int)((M + kRxScan - 1) / kRxScan);
            k_cs_hist<<<T, kRxThreads, 0, st>>>(key[0], N, T, w.rx_hist);
            k_rx_scan_sums<<<nb, 1024, 0, st>>>(w.rx_hist, M, w.rx_bsum);
            k_rx_scan_top<<<1, 1024, 0, st>>>(w.rx_bsum, nb);
            k_rx_scan_down<<<nb, 1024, 0, st>>>(w.rx_hist, M, w.rx_bsum);
            k_cs_scatter<<<T, kRxThreads, 0, st>>>(key[0], key[1], N, T, w.rx_hist, in, out);
            k_bin_offsets<<<(unsigned)((N + 1 + 255) / 256), 256, 0, st>>>(key[1], N, n_leaves, offsets);
            return cudaGetLastError();
        }
        const int passes = std::max(1, (bits + 7) / 8);
        const int T = (int)rx_tiles(N);
        const int64_t M = 256 * (int64_t)T;
        const int nb = (int)((M + kRxScan - 1) / kRxScan);
        for (int p = 0; p < passes; ++p) {
            const int src = p & 1, dst = src ^ 1;
            k_rx_hist<<<T, kRxThreads, 0, st>>>(key[src], N, 8 * p, T, w.rx_hist);
            k_rx_scan_sums<<<nb, 1024, 0, st>>>(w.rx_hist, M, w.rx_bsum);
            k_rx_scan_top<<<1, 1024, 0, st>>>(w.rx_bsum, nb);
            k_rx_scan_down<<<nb, 1024, 0, st>>>(w.rx_hist, M, w.rx_bsum);
            k_rx_scatter<<<T, kRxThreads, 0, st>>>(key[src], idx[src], key[dst], idx[dst], N, 8 * p, T, w.rx_hist);
        }
        const int fin = passes & 1;
        k_gather_idx<<<(unsigned)((N + 255) / 256), 256, 0, st>>>(N, idx[fin], in, out);
        k_bin_offsets<<<(unsigned)((N + 1 + 255) / 256), 256, 0, st>>>(key[fin], N, n_leaves, offsets);
    } else {
        k_bin_offsets<<<1, 256, 0, st>>>(key[0], 0, n_leaves, offsets);
    }
    return cudaGetLastError();
}

cudaError_t launch_kd_gather(cudaStream_t st, int64_t N, const float4* rec, const BatchDesc& in,
                             const BatchDesc& out) {
    if (N == 0) return cudaSuccess;
    k_kd_gather<<<(unsigned)((N + 255) / 256), 256, 0, st>>>(N, rec, in, out);
    return cudaGetLastError();
}

}  // namespace sdmm
