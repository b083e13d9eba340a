// kernels.h -- host-side launch helpers of the SDMM kernels (internal).
#pragma once

#include <cuda_runtime.h>

#include "common.cuh"

namespace sdmm {

enum { MODE_FIT = 0, MODE_GRAD = 1, MODE_TWO = 2 };
// new-chart records of the two-pass covariance update: floats per component
constexpr int kChart = 16;
enum { OP_CONDITION = 0, OP_SAMPLE = 1, OP_PDF = 2 };

struct GridF {
    float lo[3];
    float scale[3];
    int32_t dims[3];
    int32_t on;
};

cudaError_t launch_set_desc(cudaStream_t s, WsHeader* ws, const BatchDesc& d);
cudaError_t launch_build_chunks(cudaStream_t s, WsHeader* ws, int64_t* cb, int32_t* cr, int64_t* units,
                                int chunk, int min_samples, int64_t max_chunks);
cudaError_t launch_accumulate(cudaStream_t s, int mode, int KP, int grid, WsHeader* ws,
                              const int64_t* cb, const int32_t* cr, const float* etab, int K,
                              int chunk, int density, float* partial, int ps, int write_ll,
                              const float* chart2 = nullptr, int euclid = 0, int chart_offsets = 0);
// specialised E-step of the fit and the objective's forward pass, KP in 4..32
enum { ESTEP_CHART = 0, ESTEP_OFFSETS = 1, ESTEP_EUCLID = 2, ESTEP_SOLID = 3, ESTEP_SOLID_OFFSETS = 4,
       ESTEP_TWO = 5, ESTEP_TWO_SOLID = 6 };
bool estep_fast_supported(int KP);
cudaError_t launch_estep_fast(cudaStream_t s, int KP, int grid, WsHeader* ws, const int64_t* cb,
                              const int32_t* cr, const float* etab, int K, int chunk, float* partial,
                              int ps, int write_ll, int variant, const float* chart2 = nullptr);
// ystats: the E-step partials are in whitened coordinates (k_estep); the
// reductions take them back to the chart
cudaError_t launch_new_charts(cudaStream_t s, int64_t R, WsHeader* ws, const int64_t* cb,
                              const float* partial, int ps, const sdmm_config& cfg,
                              const sdmm_state& st, float* chart2, int ystats);
cudaError_t launch_reduce_mstep(cudaStream_t s, int64_t R, WsHeader* ws, const int64_t* cb,
                                const float* partial, int ps, const sdmm_config& cfg,
                                const sdmm_state& st, int iter, const float* xref,
                                const float* partial2 = nullptr, int ps2 = 0, int threads = 128,
                                int ystats = 0);
// contraction form on the tensor cores
size_t tc_smem_bytes(int K, int prec);

cudaError_t launch_tc_prepare(cudaStream_t s, int K, int64_t R, const sdmm_state& st, float* ctab,
                              float* xref, int euclid = 0);
int tc_ctas_per_sm(int K, int prec);
cudaError_t launch_tc_estep(cudaStream_t s, int K, int prec, int grid, WsHeader* ws, const int32_t* cr,
                            const int64_t* units, const float* ctab, const float* xref, float* partial,
                            int ps, int write_ll, int euclid = 0, int solid = 0);
cudaError_t launch_reduce_objective(cudaStream_t s, int64_t R, const WsHeader* ws,
                                    const int64_t* cb, const float* partial, int ps,
                                    const sdmm_config& cfg, const sdmm_state& st, double* F,
                                    const double* dF, float* gd, float* gL, float* ga, int ystats);
cudaError_t launch_init(cudaStream_t s, int64_t R, const sdmm_config& cfg, const BatchDesc& d,
                        const double* extent, const double* uniforms, const sdmm_state& st);
cudaError_t launch_prepare(cudaStream_t s, int K, int64_t R, const sdmm_state& st,
                           const double* logits, const double* delta, int euclid = 0);

cudaError_t launch_query(cudaStream_t s, int op, int KP, int grid, const float* qtab, int K,
                         int64_t R, int64_t Q, const float* qx, const int32_t* region,
                         const GridF& g, uint64_t seed, const float* uni, const float* dir_in,
                         float* cond_pi, float* cond_m, float* cond_L, float* dir_out,
                         float* pdf_out, uint8_t* valid_out);

// sampling / pdf with one thread per query (K <= 16); with perm, slot j
// processes query perm[j] (< 0: empty) and writes its record sorted_out[j]
cudaError_t launch_query_q(cudaStream_t s, int op, int KP, int grid, const float* qtab, int K, int64_t R,
                           int64_t Q, const float* qx, const int32_t* region, const GridF& g, const int32_t* perm,
                           float4* sorted_out, uint64_t seed, const float* uni, const float* dir_in,
                           float* dir_out, float* pdf_out, uint8_t* valid_out);
// sampling / pdf with the queries binned by region in the caller's workspace
// (K <= 16); qbin_workspace_bytes(R, Q) bytes, 256-byte aligned
size_t qbin_workspace_bytes(int64_t R, int64_t Q);
cudaError_t launch_query_binned(cudaStream_t s, int op, int KP, int grid, const float* qtab, int K, int64_t R,
                                int64_t Q, const float* qx, const int32_t* region, const GridF& g, uint64_t seed,
                                const float* uni, const float* dir_in, float* dir_out, float* pdf_out,
                                uint8_t* valid_out, void* ws);

cudaError_t launch_validate(cudaStream_t s, const BatchDesc& d, int64_t N, float tol, unsigned long long* counts,
                            int grid);
cudaError_t launch_wait_selftest(cudaStream_t s, uint64_t limit_ns, int arrive, int* status,
                                 unsigned long long* elapsed_ns);
cudaError_t launch_tc_selftest(cudaStream_t s, int kind, int N, int Kd, const float* A, const float* B,
                               float* D, int variant, int* status);

// ---- spatial kD-tree (kdtree.cu)
constexpr int kKdTile = 1024;                 // samples per tile of the refinement rounds

struct KdWork {
    float4* rec[2];              // (x, y, z, sample index as int bits), ping-pong [N]
    int64_t* seg_off[2];         // segment offsets [cap_leaves + 1]
    int32_t* seg_node[2];        // tree node of each segment
    int64_t* seg_parent[2];      // leaf of the call's input each segment descends from
    int32_t* seg_axis;
    double* seg_split;
    float* seg_split_f;          // [cap_leaves] float thresholds of seg_split
    float* split_f;              // [cap_nodes] float thresholds of the tree's splits (binning)
    int32_t* seg_flag;
    int32_t* seg_new;
    unsigned long long* seg_sum; // [cap_leaves][6]
    unsigned long long* seg_left;
    int32_t* tile_seg;           // [max_tiles]
    int64_t* tile_start;
    int32_t* tile_left;
    int64_t* tile_prefix;
    int32_t* seg_tile0;          // [cap_leaves + 2] first tile of each segment
    int32_t* counters;           // [0] tiles, [1] splits
    uint32_t* rx_hist;           // binning: digit counts per radix tile, then their offsets
    uint32_t* rx_bsum;           // binning: scan block sums
    int64_t max_tiles;
};
cudaError_t launch_kd_grid(cudaStream_t s, int levels, int32_t* axis, double* split, int32_t* left, int32_t* leaf);
cudaError_t launch_kd_lookup(cudaStream_t s, const int32_t* axis, const double* split, const int32_t* left,
                             const int32_t* leaf, int max_depth, int64_t Q, const float* px, const float* py,
                             const float* pz, int32_t* out);
cudaError_t launch_kd_prepare(cudaStream_t st, const KdWork& w, const int32_t* tree_axis,
                              const int32_t* tree_leaf, int32_t n_nodes, int32_t S0, const int64_t* offsets_in,
                              int64_t N, const float* px, const float* py, const float* pz);
cudaError_t kd_rounds(cudaStream_t st, const KdWork& w, int64_t c, int32_t* tree_axis,
                      double* tree_split, int32_t* tree_left, int32_t* tree_leaf, int32_t* n_nodes,
                      int32_t* n_leaves, int32_t cap_nodes, int32_t cap_leaves, int32_t S0, int64_t N,
                      const float4** rec_final,
                      int64_t** seg_off_final, int64_t** seg_parent_final, int32_t* S_final, int* overflow);
int64_t rx_tiles(int64_t N);
int64_t rx_hist_entries(int64_t N);
int64_t rx_scan_blocks(int64_t N);
cudaError_t launch_kd_bin(cudaStream_t st, const KdWork& w, const int32_t* axis, const double* split,
                          const int32_t* left, const int32_t* leaf, int32_t n_nodes, int32_t n_leaves, int64_t N,
                          const float* px, const float* py, const float* pz, const BatchDesc& in,
                          const BatchDesc& out, int64_t* offsets);
cudaError_t launch_kd_gather(cudaStream_t st, int64_t N, const float4* rec, const BatchDesc& in,
                             const BatchDesc& out);
cudaError_t launch_gather_state(cudaStream_t s, int K, int64_t R_out, const int64_t* src, const sdmm_state& in,
                                const sdmm_state& out);

// ---- product sampling with a BSDF mixture (product.cu)
cudaError_t launch_product(cudaStream_t s, int op, int KP, int grid, const float* qtab, int K, int64_t R, int64_t Q,
                           const float* qx, const int32_t* region, const GridF& g, const float* bw, const float* bmu,
                           const float* bL, int J, uint64_t seed, const float* uni, const float* dir_in, float* dout,
                           float* pout, uint8_t* vout);

}  // namespace sdmm
