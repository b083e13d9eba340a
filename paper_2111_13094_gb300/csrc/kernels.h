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
                              const float* chart2 = nullptr);
cudaError_t launch_new_charts(cudaStream_t s, int64_t R, WsHeader* ws, const int64_t* cb,
                              const float* partial, int ps, const sdmm_config& cfg,
                              const sdmm_state& st, float* chart2);
cudaError_t launch_reduce_mstep(cudaStream_t s, int64_t R, WsHeader* ws, const int64_t* cb,
                                const float* partial, int ps, const sdmm_config& cfg,
                                const sdmm_state& st, int iter, const float* xref,
                                const float* partial2 = nullptr, int ps2 = 0);
// contraction form on the tensor cores
size_t tc_smem_bytes(int K, int prec);

cudaError_t launch_tc_prepare(cudaStream_t s, int K, int64_t R, const sdmm_state& st, float* ctab,
                              float* xref);
int tc_ctas_per_sm(int K, int prec);
cudaError_t launch_tc_estep(cudaStream_t s, int K, int prec, int grid, WsHeader* ws, const int32_t* cr,
                            const int64_t* units, const float* ctab, const float* xref, float* partial,
                            int ps, int write_ll);
cudaError_t launch_reduce_objective(cudaStream_t s, int64_t R, const WsHeader* ws,
                                    const int64_t* cb, const float* partial, int ps,
                                    const sdmm_config& cfg, const sdmm_state& st, double* F,
                                    const double* dF, float* gd, float* gL, float* ga);
cudaError_t launch_init(cudaStream_t s, int64_t R, const sdmm_config& cfg, const BatchDesc& d,
                        const double* extent, const double* uniforms, const sdmm_state& st);
cudaError_t launch_prepare(cudaStream_t s, int K, int64_t R, const sdmm_state& st,
                           const double* logits, const double* delta);

cudaError_t launch_query(cudaStream_t s, int op, int KP, int grid, const float* qtab, int K,
                         int64_t R, int64_t Q, const float* qx, const int32_t* region,
                         const GridF& g, uint64_t seed, const float* uni, const float* dir_in,
                         float* cond_pi, float* cond_m, float* cond_L, float* dir_out,
                         float* pdf_out, uint8_t* valid_out);

cudaError_t launch_tc_selftest(cudaStream_t s, int kind, int N, int Kd, const float* A, const float* B,
                               float* D, int variant, int* status);

}  // namespace sdmm
