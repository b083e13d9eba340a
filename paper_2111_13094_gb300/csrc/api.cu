// api.cu -- the C ABI of include/sdmm.h: argument checks, workspace layout,
// kernel launch sequences, CUDA-graph fit plans and the autotuner.
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <mutex>
#include <vector>

#include "common.cuh"
#include "kernels.h"

using namespace sdmm;

namespace {

thread_local char g_err[512] = "";

// SDMM_PROFILE=1 (environment): the main entry points record CUDA events
// around their launches on their stream, wait for them and print
// "sdmm: <call> <ms> ms" to stderr.  The calls are then synchronous; streams
// that are being captured into a graph are left alone.
bool profile_on() {
    static const bool on = [] {
        const char* v = std::getenv("SDMM_PROFILE");
        return v != nullptr && v[0] != '\0' && v[0] != '0';
    }();
    return on;
}

struct ProfileScope {
    const char* name;
    cudaStream_t s;
    cudaEvent_t a = nullptr, b = nullptr;
    ProfileScope(const char* n, sdmm_stream st) : name(n), s(static_cast<cudaStream_t>(st)) {
        if (!profile_on()) return;
        cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
        if (cudaStreamIsCapturing(s, &cs) != cudaSuccess || cs != cudaStreamCaptureStatusNone) {
            cudaGetLastError();
            return;
        }
        if (cudaEventCreate(&a) != cudaSuccess || cudaEventCreate(&b) != cudaSuccess) {
            if (a) cudaEventDestroy(a);
            a = b = nullptr;
            cudaGetLastError();
            return;
        }
        cudaEventRecord(a, s);
    }
    ~ProfileScope() {
        if (!a) return;
        cudaEventRecord(b, s);
        float ms = 0.f;
        if (cudaEventSynchronize(b) == cudaSuccess && cudaEventElapsedTime(&ms, a, b) == cudaSuccess)
            std::fprintf(stderr, "sdmm: %s %.3f ms\n", name, ms);
        cudaGetLastError();
        cudaEventDestroy(a);
        cudaEventDestroy(b);
    }
};

sdmm_status fail(sdmm_status code, const char* fmt, ...) {
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_err, sizeof(g_err), fmt, ap);
    va_end(ap);
    return code;
}

sdmm_status cuda_fail(cudaError_t e, const char* what) {
    return fail(SDMM_ERR_CUDA, "%s: %s", what, cudaGetErrorString(e));
}

#define SDMM_CUDA(call, what)                          \
    do {                                               \
        cudaError_t e_ = (call);                       \
        if (e_ != cudaSuccess) return cuda_fail(e_, what); \
    } while (0)

int pow2_ceil(int K) {
    int p = 1;
    while (p < K) p <<= 1;
    return p;
}

int sm_count() {
    int dev = 0, n = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return 0;
    if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return 0;
    return n;
}

constexpr size_t kAlign = 256;
size_t align_up(size_t x) { return (x + kAlign - 1) / kAlign * kAlign; }

sdmm_status check_config(const sdmm_config* cfg) {
    if (!cfg) return fail(SDMM_ERR_INVALID_ARG, "config is NULL");
    if (cfg->K < 1) return fail(SDMM_ERR_INVALID_ARG, "K = %d must be >= 1", cfg->K);
    if (cfg->K > SDMM_MAX_K) return fail(SDMM_ERR_UNSUPPORTED, "K = %d > %d", cfg->K, SDMM_MAX_K);
    if (cfg->min_samples < 1) return fail(SDMM_ERR_INVALID_ARG, "min_samples must be >= 1");
    if (cfg->eta_mode != SDMM_ETA_ROBBINS_MONRO && cfg->eta_mode != SDMM_ETA_ONE)
        return fail(SDMM_ERR_INVALID_ARG, "eta_mode %d", cfg->eta_mode);
    if (cfg->estep_density != SDMM_DENSITY_TANGENT && cfg->estep_density != SDMM_DENSITY_SOLID_ANGLE)
        return fail(SDMM_ERR_INVALID_ARG, "estep_density %d", cfg->estep_density);
    if (cfg->prior_scale_mode != SDMM_PRIOR_SCALE_SEEN && cfg->prior_scale_mode != SDMM_PRIOR_SCALE_ARRAY)
        return fail(SDMM_ERR_INVALID_ARG, "prior_scale_mode %d", cfg->prior_scale_mode);
    if (cfg->precision < SDMM_PREC_FP32 || cfg->precision > SDMM_PREC_TC_6XBF16)
        return fail(SDMM_ERR_INVALID_ARG, "precision %d", cfg->precision);
    if (cfg->precision != SDMM_PREC_FP32 && !(cfg->K == 16 || cfg->K == 32))
        return fail(SDMM_ERR_UNSUPPORTED, "tensor-core precision needs K = 16 or 32 (K = %d)", cfg->K);
    if (cfg->chunk != 0 && (cfg->chunk < 256 || cfg->chunk > 65536 || cfg->chunk % 256 != 0))
        return fail(SDMM_ERR_INVALID_ARG, "chunk %d: 0 or a multiple of 256 in [256, 65536]", cfg->chunk);
    if (cfg->ctas_per_sm < 0 || cfg->ctas_per_sm > 4)
        return fail(SDMM_ERR_INVALID_ARG, "ctas_per_sm %d: 0..4", cfg->ctas_per_sm);
    if (cfg->cov_update != SDMM_COV_FIRST_ORDER && cfg->cov_update != SDMM_COV_TWO_PASS)
        return fail(SDMM_ERR_INVALID_ARG, "cov_update %d", cfg->cov_update);
    if (cfg->cov_update == SDMM_COV_TWO_PASS && cfg->precision != SDMM_PREC_FP32)
        return fail(SDMM_ERR_UNSUPPORTED, "the two-pass covariance update runs on the FP32 SIMT path");
    if (cfg->cov_update == SDMM_COV_TWO_PASS && cfg->eta_mode != SDMM_ETA_ONE)
        return fail(SDMM_ERR_UNSUPPORTED, "the two-pass covariance update is defined for eta_mode = ETA_ONE");
    if (cfg->dir_coords != SDMM_DIR_TANGENT && cfg->dir_coords != SDMM_DIR_EUCLIDEAN)
        return fail(SDMM_ERR_INVALID_ARG, "dir_coords %d", cfg->dir_coords);
    if (cfg->dir_coords == SDMM_DIR_EUCLIDEAN && cfg->cov_update == SDMM_COV_TWO_PASS)
        return fail(SDMM_ERR_UNSUPPORTED, "the two-pass covariance update needs tangent charts");
    if (cfg->dir_coords == SDMM_DIR_EUCLIDEAN && cfg->precision != SDMM_PREC_FP32 &&
        cfg->precision != SDMM_PREC_TC_6XBF16 && cfg->precision != SDMM_PREC_TC_3XTF32)
        return fail(SDMM_ERR_UNSUPPORTED, "the Euclidean ablation runs on FP32 SIMT, 6xBF16 or 3xTF32");
    const double v[6] = {cfg->eta_alpha, cfg->eta_beta, cfg->prior_q, cfg->prior_a,
                         cfg->prior_B_pos, cfg->prior_B_dir};
    for (double x : v)
        if (!std::isfinite(x) || x < 0.0) return fail(SDMM_ERR_INVALID_ARG, "prior/eta constants must be finite and >= 0");
    return SDMM_OK;
}

sdmm_status check_state(const sdmm_state* st, bool fit) {
    if (!st) return fail(SDMM_ERR_INVALID_ARG, "state is NULL");
    if (!st->pi || !st->mu_x || !st->mu_w || !st->L || !st->etab || !st->qtab)
        return fail(SDMM_ERR_INVALID_ARG, "state parameter/table pointers must be non-NULL");
    if (fit && (!st->S0 || !st->S2 || !st->Wbar || !st->n_seen || !st->step_j || !st->status))
        return fail(SDMM_ERR_INVALID_ARG, "state statistics pointers must be non-NULL");
    if ((reinterpret_cast<uintptr_t>(st->etab) | reinterpret_cast<uintptr_t>(st->qtab)) & 15u)
        return fail(SDMM_ERR_INVALID_ARG, "etab/qtab must be 16-byte aligned");
    return SDMM_OK;
}

sdmm_status check_samples(const sdmm_samples* s) {
    if (!s) return fail(SDMM_ERR_INVALID_ARG, "samples is NULL");
    if (s->R < 1 || s->R > (int64_t)INT32_MAX / 2) return fail(SDMM_ERR_INVALID_ARG, "R = %lld", (long long)s->R);
    if (s->N < 0) return fail(SDMM_ERR_INVALID_ARG, "N = %lld", (long long)s->N);
    if (!s->offsets) return fail(SDMM_ERR_INVALID_ARG, "offsets is NULL");
    const float* p[7] = {s->px, s->py, s->pz, s->ox, s->oy, s->oz, s->w};
    for (int i = 0; i < 7; ++i) {
        if (s->N > 0 && !p[i]) return fail(SDMM_ERR_INVALID_ARG, "sample stream %d is NULL", i);
        if (reinterpret_cast<uintptr_t>(p[i]) & 3u) return fail(SDMM_ERR_INVALID_ARG, "sample stream %d misaligned", i);
    }
    return SDMM_OK;
}

int default_ctas(const sdmm_config* cfg) { return cfg->ctas_per_sm > 0 ? cfg->ctas_per_sm : 2; }

int choose_chunk(const sdmm_config* cfg, int64_t N) {
    if (cfg->chunk > 0) return cfg->chunk;
    const int64_t G = (int64_t)std::max(1, sm_count()) * default_ctas(cfg);
    int64_t c = 256;
    while (c < 4096 && c * G * 16 < N) c <<= 1;
    return (int)c;
}

struct Layout {
    size_t header, chunk_base, chunk_region, partial, ctab, xref, units, chart2, partial2, total;
    int chunk, ps, ps2;
    int64_t max_chunks;
};

bool tensor_core(const sdmm_config* cfg) { return cfg->precision != SDMM_PREC_FP32; }

Layout layout(const sdmm_config* cfg, int64_t R, int64_t N, int chunk) {
    Layout L{};
    L.chunk = chunk;
    // tensor-core partials hold 3K feature-space rows of 28 and four per-quadrant
    // (W, sum w l) pairs, the SIMT ones 21K statistics
    L.ps = tensor_core(cfg) ? ((3 * cfg->K * kFeat + 8) + 3) & ~3 : partial_stride(cfg->K);
    L.max_chunks = (N + chunk - 1) / chunk + R;
    size_t o = 0;
    L.header = o;
    o = align_up(o + sizeof(WsHeader));
    L.chunk_base = o;
    o = align_up(o + sizeof(int64_t) * (size_t)(R + 1));
    L.chunk_region = o;
    o = align_up(o + sizeof(int32_t) * (size_t)L.max_chunks);
    L.partial = o;
    o = align_up(o + sizeof(float) * (size_t)L.max_chunks * L.ps);
    L.ctab = L.xref = L.units = o;
    if (tensor_core(cfg)) {
        L.ctab = o;
        o = align_up(o + sizeof(float) * (size_t)R * cfg->K * 6 * 32);
        L.xref = o;
        o = align_up(o + sizeof(float) * (size_t)R * 4);
        L.units = o;
        o = align_up(o + sizeof(int64_t) * 2 * (size_t)L.max_chunks);
    }
    L.chart2 = L.partial2 = o;
    L.ps2 = 0;
    if (cfg->cov_update == SDMM_COV_TWO_PASS) {   // second pass: new charts and their moments
        L.ps2 = ((15 * cfg->K) + 3) & ~3;
        L.chart2 = o;
        o = align_up(o + sizeof(float) * (size_t)R * cfg->K * kChart);
        L.partial2 = o;
        o = align_up(o + sizeof(float) * (size_t)L.max_chunks * L.ps2);
    }
    L.total = o;
    return L;
}

struct WsPtrs {
    WsHeader* hdr;
    int64_t* cb;
    int32_t* cr;
    float* partial;
    float* ctab;
    float* xref;
    int64_t* units;     // tensor-core path only, else null
    float* chart2;      // two-pass covariance update only, else null
    float* partial2;
};

WsPtrs ws_ptrs(void* ws, const Layout& L) {
    char* b = static_cast<char*>(ws);
    return WsPtrs{reinterpret_cast<WsHeader*>(b + L.header), reinterpret_cast<int64_t*>(b + L.chunk_base),
                  reinterpret_cast<int32_t*>(b + L.chunk_region), reinterpret_cast<float*>(b + L.partial),
                  reinterpret_cast<float*>(b + L.ctab), reinterpret_cast<float*>(b + L.xref),
                  L.units < L.total ? reinterpret_cast<int64_t*>(b + L.units) : nullptr,
                  L.ps2 ? reinterpret_cast<float*>(b + L.chart2) : nullptr,
                  L.ps2 ? reinterpret_cast<float*>(b + L.partial2) : nullptr};
}

sdmm_status check_ws(void* ws, size_t bytes, const Layout& L) {
    if (!ws) return fail(SDMM_ERR_INVALID_ARG, "workspace is NULL");
    if (reinterpret_cast<uintptr_t>(ws) % kAlign) return fail(SDMM_ERR_INVALID_ARG, "workspace must be 256-byte aligned");
    if (bytes < L.total)
        return fail(SDMM_ERR_WORKSPACE, "workspace %zu bytes < required %zu", bytes, L.total);
    return SDMM_OK;
}

BatchDesc make_desc(const sdmm_samples* s, const double* prior, float* loglik) {
    BatchDesc d{};
    d.p[0] = s->px; d.p[1] = s->py; d.p[2] = s->pz;
    d.p[3] = s->ox; d.p[4] = s->oy; d.p[5] = s->oz; d.p[6] = s->w;
    d.offsets = s->offsets;
    d.R = s->R;
    d.N = s->N;
    d.prior_scale = prior;
    d.loglik = loglik;
    return d;
}

// The per-step launch sequence of a fit (shared by direct calls and plans).
struct FitLaunch {
    sdmm_config cfg;
    sdmm_state st;
    Layout L;
    WsPtrs w;
    int64_t R;
    int iters;
    int grid;
    int want_ll;
};

sdmm_status enqueue_fit(const FitLaunch& f, cudaStream_t s, std::vector<cudaEvent_t>* evs) {
    const int KP = pow2_ceil(f.cfg.K);
    const bool tcore = tensor_core(&f.cfg);
    const int euclid = f.cfg.dir_coords == SDMM_DIR_EUCLIDEAN;
    const int mstep_threads = f.R > 3 * (int64_t)std::max(1, sm_count()) ? 32 : 128;
    // the specialised E-step leaves its statistics in whitened coordinates
    const int ystats = !tcore && estep_fast_supported(KP);
    SDMM_CUDA(launch_build_chunks(s, f.w.hdr, f.w.cb, f.w.cr, f.w.units, f.L.chunk, f.cfg.min_samples,
                                  f.L.max_chunks),
              "build_chunks");
    for (int it = 0; it < f.iters; ++it) {
        const int wll = f.want_ll && it == f.iters - 1;
        if (tcore)
            SDMM_CUDA(launch_tc_prepare(s, f.cfg.K, f.R, f.st, f.w.ctab, f.w.xref, euclid), "tc_prepare");
        if (evs) SDMM_CUDA(cudaEventRecordWithFlags((*evs)[2 * it], s, cudaEventRecordExternal), "event");
        if (tcore) {
            const int grid = std::max(1, sm_count()) * tc_ctas_per_sm(f.cfg.K, f.cfg.precision);   // persistent
            SDMM_CUDA(launch_tc_estep(s, f.cfg.K, f.cfg.precision, grid, f.w.hdr, f.w.cr, f.w.units, f.w.ctab,
                                      f.w.xref, f.w.partial, f.L.ps, wll, euclid,
                                      f.cfg.estep_density == SDMM_DENSITY_SOLID_ANGLE),
                      "tc_estep");
        } else {
            SDMM_CUDA(launch_accumulate(s, MODE_FIT, KP, f.grid, f.w.hdr, f.w.cb, f.w.cr, f.st.etab, f.cfg.K,
                                        f.L.chunk, f.cfg.estep_density, f.w.partial, f.L.ps, wll, nullptr,
                                        euclid),
                      "accumulate");
        }
        if (evs) SDMM_CUDA(cudaEventRecordWithFlags((*evs)[2 * it + 1], s, cudaEventRecordExternal), "event");
        if (f.w.partial2 != nullptr) {   // accurate covariance update: second pass in the new charts
            SDMM_CUDA(launch_new_charts(s, f.R, f.w.hdr, f.w.cb, f.w.partial, f.L.ps, f.cfg, f.st, f.w.chart2,
                                        ystats),
                      "new_charts");
            SDMM_CUDA(launch_accumulate(s, MODE_TWO, KP, f.grid, f.w.hdr, f.w.cb, f.w.cr,
                                        f.st.etab, f.cfg.K, f.L.chunk, f.cfg.estep_density, f.w.partial2,
                                        f.L.ps2, 0, f.w.chart2),
                      "accumulate_two");
        }
        SDMM_CUDA(launch_reduce_mstep(s, f.R, f.w.hdr, f.w.cb, f.w.partial, f.L.ps, f.cfg, f.st, it,
                                      tcore ? f.w.xref : nullptr, f.w.partial2, f.L.ps2, mstep_threads, ystats),
                  "reduce_mstep");
    }
    return SDMM_OK;
}

}  // namespace

// ===========================================================================
// Fixed scratch of sdmm_fit_regions_noalloc, for callers that may not
// allocate device memory (see include/sdmm.h).  It is part of this library's
// device image, so every GPU that loads the library holds it until exit.
static __device__ __align__(256) unsigned char g_noalloc_scratch[SDMM_NOALLOC_SCRATCH_BYTES];

namespace {

constexpr int kMaxDevices = 64;
std::mutex g_noalloc_mu;
void* g_noalloc_ptr[kMaxDevices] = {};

// Device address of the fixed scratch on the current device.  In host code the
// array's name is only a host-side stand-in, so the address is looked up once
// per device, with that device current, and cached.
sdmm_status noalloc_scratch(void** out) {
    int dev = -1;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGetDevice");
    if (dev < 0 || dev >= kMaxDevices) return fail(SDMM_ERR_UNSUPPORTED, "device ordinal %d", dev);
    std::lock_guard<std::mutex> lock(g_noalloc_mu);
    if (g_noalloc_ptr[dev] == nullptr) {
        void* p = nullptr;
        e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess) return cuda_fail(e, "cudaGetSymbolAddress of the fixed scratch");
        g_noalloc_ptr[dev] = p;
    }
    *out = g_noalloc_ptr[dev];
    return SDMM_OK;
}

}  // namespace

extern "C" {

void sdmm_config_default(sdmm_config* cfg, int32_t K) {
    if (!cfg) return;
    std::memset(cfg, 0, sizeof(*cfg));
    cfg->K = K;
    cfg->min_samples = 16;                 // Sec. 4.2
    cfg->eta_mode = SDMM_ETA_ROBBINS_MONRO;
    cfg->estep_density = SDMM_DENSITY_TANGENT;
    cfg->prior_scale_mode = SDMM_PRIOR_SCALE_SEEN;
    cfg->precision = SDMM_PREC_FP32;
    cfg->chunk = 0;
    cfg->ctas_per_sm = 0;
    cfg->eta_alpha = 0.5;                  // Sec. 4.3
    cfg->eta_beta = 0.1;
    cfg->prior_q = 1.0;                    // q = 1/K
    cfg->prior_a = 5.0;                    // a = 5/K
    cfg->prior_B_pos = 1e-4;               // B = a diag(0.1, 0.1, 1, 1, 1) 1e-4
    cfg->prior_B_dir = 1e-5;
}

const char* sdmm_last_error(void) { return g_err; }

const char* sdmm_version(void) { return "sdmm-gb300 0.1 (sm_103a)"; }

sdmm_status sdmm_fit_workspace_size(const sdmm_config* cfg, int64_t R, int64_t N, size_t* bytes) {
    sdmm_status e = check_config(cfg);
    if (e) return e;
    if (!bytes) return fail(SDMM_ERR_INVALID_ARG, "bytes is NULL");
    if (R < 1 || N < 0) return fail(SDMM_ERR_INVALID_ARG, "R = %lld, N = %lld", (long long)R, (long long)N);
    *bytes = layout(cfg, R, N, choose_chunk(cfg, N)).total;
    return SDMM_OK;
}

sdmm_status sdmm_init_regions(const sdmm_config* cfg, const sdmm_samples* s, const double* extent,
                              const double* uniforms, sdmm_state* st, sdmm_stream stream) {
    ProfileScope prof_("init_regions", stream);
    sdmm_status e;
    if ((e = check_config(cfg)) || (e = check_samples(s)) || (e = check_state(st, true))) return e;
    if (!extent || !uniforms) return fail(SDMM_ERR_INVALID_ARG, "extent/uniforms are NULL");
    SDMM_CUDA(launch_init(stream, s->R, *cfg, make_desc(s, nullptr, nullptr), extent, uniforms, *st),
              "init_regions");
    return SDMM_OK;
}

sdmm_status sdmm_fit_regions(const sdmm_config* cfg, const sdmm_samples* s, int32_t iters,
                             const double* prior_scale, sdmm_state* st, float* loglik_out,
                             void* workspace, size_t ws_bytes, sdmm_stream stream) {
    ProfileScope prof_("fit_regions", stream);
    sdmm_status e;
    if ((e = check_config(cfg)) || (e = check_samples(s)) || (e = check_state(st, true))) return e;
    if (iters < 1) return fail(SDMM_ERR_INVALID_ARG, "iters = %d must be >= 1", iters);
    if (cfg->prior_scale_mode == SDMM_PRIOR_SCALE_ARRAY && !prior_scale)
        return fail(SDMM_ERR_INVALID_ARG, "prior_scale_mode ARRAY needs prior_scale");
    const Layout L = layout(cfg, s->R, s->N, choose_chunk(cfg, s->N));
    if ((e = check_ws(workspace, ws_bytes, L))) return e;
    const int nsm = sm_count();
    if (nsm <= 0) return fail(SDMM_ERR_CUDA, "no CUDA device");
    FitLaunch f{*cfg, *st, L, ws_ptrs(workspace, L), s->R, iters, nsm * default_ctas(cfg),
                loglik_out != nullptr};
    SDMM_CUDA(launch_set_desc(stream, f.w.hdr, make_desc(s, prior_scale, loglik_out)), "set_desc");
    return enqueue_fit(f, stream, nullptr);
}

sdmm_status sdmm_prepare(const sdmm_config* cfg, int64_t R, sdmm_state* st, const double* logits,
                         const double* delta, sdmm_stream stream) {
    ProfileScope prof_("prepare", stream);
    sdmm_status e;
    if ((e = check_config(cfg)) || (e = check_state(st, false))) return e;
    if (R < 1) return fail(SDMM_ERR_INVALID_ARG, "R = %lld", (long long)R);
    SDMM_CUDA(launch_prepare(stream, cfg->K, R, *st, logits, delta, cfg->dir_coords == SDMM_DIR_EUCLIDEAN),
              "prepare");
    return SDMM_OK;
}

// ---------------------------------------------------------------- queries
static sdmm_status query_common(const sdmm_config* cfg, const sdmm_state* st, int64_t R, int64_t Q,
                                const float* qx, const int32_t* region, const sdmm_grid* grid,
                                GridF* g) {
    sdmm_status e;
    if ((e = check_config(cfg)) || (e = check_state(st, false))) return e;
    if (cfg->dir_coords != SDMM_DIR_TANGENT)
        return fail(SDMM_ERR_UNSUPPORTED, "queries need tangent charts (dir_coords = SDMM_DIR_TANGENT)");
    if (R < 1 || Q < 0) return fail(SDMM_ERR_INVALID_ARG, "R = %lld, Q = %lld", (long long)R, (long long)Q);
    if (Q > 0 && !qx) return fail(SDMM_ERR_INVALID_ARG, "qx is NULL");
    std::memset(g, 0, sizeof(*g));
    if (!region) {
        if (!grid) return fail(SDMM_ERR_INVALID_ARG, "need region ids or a grid");
        int64_t cells = 1;
        for (int c = 0; c < 3; ++c) {
            if (grid->dims[c] < 1) return fail(SDMM_ERR_INVALID_ARG, "grid dims must be >= 1");
            if (!(grid->hi[c] > grid->lo[c])) return fail(SDMM_ERR_INVALID_ARG, "grid hi must exceed lo");
            g->lo[c] = grid->lo[c];
            g->scale[c] = (float)grid->dims[c] / (grid->hi[c] - grid->lo[c]);
            g->dims[c] = grid->dims[c];
            cells *= grid->dims[c];
        }
        if (cells > R) return fail(SDMM_ERR_INVALID_ARG, "grid has %lld cells > R", (long long)cells);
        g->on = 1;
    }
    return SDMM_OK;
}

static int query_grid(int64_t Q) {
    const int nsm = std::max(1, sm_count());
    const int64_t groups = (Q + 31) / 32;             // one warp per 32 queries at a time
    const int64_t ctas = (groups + 7) / 8;
    return (int)std::max<int64_t>(1, std::min<int64_t>(ctas, (int64_t)nsm * 8));
}

sdmm_status sdmm_condition(const sdmm_config* cfg, const sdmm_state* st, int64_t R, int64_t Q,
                           const float* qx, const int32_t* region, const sdmm_grid* grid,
                           float* cond_pi, float* cond_m, float* cond_L, sdmm_stream stream) {
    ProfileScope prof_("condition", stream);
    GridF g;
    sdmm_status e = query_common(cfg, st, R, Q, qx, region, grid, &g);
    if (e) return e;
    if (Q > 0 && (!cond_pi || !cond_m || !cond_L)) return fail(SDMM_ERR_INVALID_ARG, "outputs are NULL");
    if (Q == 0) return SDMM_OK;
    SDMM_CUDA(launch_query(stream, OP_CONDITION, pow2_ceil(cfg->K), query_grid(Q), st->qtab, cfg->K, R, Q,
                           qx, region, g, 0, nullptr, nullptr, cond_pi, cond_m, cond_L, nullptr,
                           nullptr, nullptr),
              "condition");
    return SDMM_OK;
}

sdmm_status sdmm_sample(const sdmm_config* cfg, const sdmm_state* st, int64_t R, int64_t Q,
                        const float* qx, const int32_t* region, const sdmm_grid* grid, uint64_t seed,
                        const float* uniforms, float* dir_out, float* pdf_out, uint8_t* valid_out,
                        sdmm_stream stream) {
    ProfileScope prof_("sample", stream);
    GridF g;
    sdmm_status e = query_common(cfg, st, R, Q, qx, region, grid, &g);
    if (e) return e;
    if (Q > 0 && (!dir_out || !pdf_out || !valid_out)) return fail(SDMM_ERR_INVALID_ARG, "outputs are NULL");
    if (Q == 0) return SDMM_OK;
    SDMM_CUDA(launch_query(stream, OP_SAMPLE, pow2_ceil(cfg->K), query_grid(Q), st->qtab, cfg->K, R, Q, qx,
                           region, g, seed, uniforms, nullptr, nullptr, nullptr, nullptr, dir_out,
                           pdf_out, valid_out),
              "sample");
    return SDMM_OK;
}

sdmm_status sdmm_query_workspace_size(int64_t R, int64_t Q, size_t* bytes) {
    if (!bytes) return fail(SDMM_ERR_INVALID_ARG, "bytes is NULL");
    if (R < 1 || Q < 0) return fail(SDMM_ERR_INVALID_ARG, "R = %lld, Q = %lld", (long long)R, (long long)Q);
    *bytes = qbin_workspace_bytes(R, Q);
    return SDMM_OK;
}

static sdmm_status binned_checks(const sdmm_config* cfg, int64_t R, int64_t Q, void* ws, size_t ws_bytes) {
    if (Q > (int64_t)INT32_MAX) return fail(SDMM_ERR_INVALID_ARG, "Q = %lld must be below 2^31", (long long)Q);
    if (R >= (int64_t)INT32_MAX) return fail(SDMM_ERR_INVALID_ARG, "R = %lld must be below 2^31", (long long)R);
    if (pow2_ceil(cfg->K) > 16) return SDMM_OK;          // processed in the given order, no workspace
    const size_t need = qbin_workspace_bytes(R, Q);
    if (!ws || (reinterpret_cast<uintptr_t>(ws) & 255u) || ws_bytes < need)
        return fail(SDMM_ERR_WORKSPACE, "query workspace must be 256-byte aligned device memory of %zu bytes", need);
    return SDMM_OK;
}

sdmm_status sdmm_sample_binned(const sdmm_config* cfg, const sdmm_state* st, int64_t R, int64_t Q,
                               const float* qx, const int32_t* region, const sdmm_grid* grid, uint64_t seed,
                               const float* uniforms, float* dir_out, float* pdf_out, uint8_t* valid_out,
                               void* workspace, size_t ws_bytes, sdmm_stream stream) {
    ProfileScope prof_("sample_binned", stream);
    GridF g;
    sdmm_status e = query_common(cfg, st, R, Q, qx, region, grid, &g);
    if (e) return e;
    if (Q > 0 && (!dir_out || !pdf_out || !valid_out)) return fail(SDMM_ERR_INVALID_ARG, "outputs are NULL");
    if ((e = binned_checks(cfg, R, Q, workspace, ws_bytes))) return e;
    if (Q == 0) return SDMM_OK;
    const int KP = pow2_ceil(cfg->K);
    if (KP > 16)
        SDMM_CUDA(launch_query(stream, OP_SAMPLE, KP, query_grid(Q), st->qtab, cfg->K, R, Q, qx, region, g, seed,
                               uniforms, nullptr, nullptr, nullptr, nullptr, dir_out, pdf_out, valid_out),
                  "sample_binned");
    else
        SDMM_CUDA(launch_query_binned(stream, OP_SAMPLE, KP, query_grid(Q), st->qtab, cfg->K, R, Q, qx, region, g,
                                      seed, uniforms, nullptr, dir_out, pdf_out, valid_out, workspace),
                  "sample_binned");
    return SDMM_OK;
}

sdmm_status sdmm_pdf_binned(const sdmm_config* cfg, const sdmm_state* st, int64_t R, int64_t Q, const float* qx,
                            const int32_t* region, const sdmm_grid* grid, const float* dir, float* pdf_out,
                            void* workspace, size_t ws_bytes, sdmm_stream stream) {
    ProfileScope prof_("pdf_binned", stream);
    GridF g;
    sdmm_status e = query_common(cfg, st, R, Q, qx, region, grid, &g);
    if (e) return e;
    if (Q > 0 && (!dir || !pdf_out)) return fail(SDMM_ERR_INVALID_ARG, "dir/pdf_out are NULL");
    if ((e = binned_checks(cfg, R, Q, workspace, ws_bytes))) return e;
    if (Q == 0) return SDMM_OK;
    const int KP = pow2_ceil(cfg->K);
    if (KP > 16)
        SDMM_CUDA(launch_query(stream, OP_PDF, KP, query_grid(Q), st->qtab, cfg->K, R, Q, qx, region, g, 0, nullptr,
                               dir, nullptr, nullptr, nullptr, nullptr, pdf_out, nullptr),
                  "pdf_binned");
    else
        SDMM_CUDA(launch_query_binned(stream, OP_PDF, KP, query_grid(Q), st->qtab, cfg->K, R, Q, qx, region, g, 0,
                                      nullptr, dir, nullptr, pdf_out, nullptr, workspace),
                  "pdf_binned");
    return SDMM_OK;
}

static sdmm_status bsdf_check(const sdmm_bsdf_lobes* b, int64_t Q) {
    if (!b) return fail(SDMM_ERR_INVALID_ARG, "bsdf is NULL");
    if (b->J < 1 || b->J > 8) return fail(SDMM_ERR_INVALID_ARG, "J = %d BSDF lobes: 1..8", b->J);
    if (Q > 0 && (!b->w || !b->mu || !b->L)) return fail(SDMM_ERR_INVALID_ARG, "BSDF arrays are NULL");
    return SDMM_OK;
}

sdmm_status sdmm_product_sample(const sdmm_config* cfg, const sdmm_state* st, int64_t R, int64_t Q,
                                const float* qx, const int32_t* region, const sdmm_grid* grid,
                                const sdmm_bsdf_lobes* bsdf, uint64_t seed, const float* uniforms,
                                float* dir_out, float* pdf_out, uint8_t* valid_out, sdmm_stream stream) {
    ProfileScope prof_("product_sample", stream);
    GridF g;
    sdmm_status e = query_common(cfg, st, R, Q, qx, region, grid, &g);
    if (!e) e = bsdf_check(bsdf, Q);
    if (e) return e;
    if (Q > 0 && (!dir_out || !pdf_out || !valid_out)) return fail(SDMM_ERR_INVALID_ARG, "outputs are NULL");
    if (Q == 0) return SDMM_OK;
    SDMM_CUDA(launch_product(stream, OP_SAMPLE, pow2_ceil(cfg->K), query_grid(Q), st->qtab, cfg->K, R, Q, qx, region,
                             g, bsdf->w, bsdf->mu, bsdf->L, bsdf->J, seed, uniforms, nullptr, dir_out, pdf_out,
                             valid_out),
              "product_sample");
    return SDMM_OK;
}

sdmm_status sdmm_product_pdf(const sdmm_config* cfg, const sdmm_state* st, int64_t R, int64_t Q, const float* qx,
                             const int32_t* region, const sdmm_grid* grid, const sdmm_bsdf_lobes* bsdf,
                             const float* dir, float* pdf_out, sdmm_stream stream) {
    ProfileScope prof_("product_pdf", stream);
    GridF g;
    sdmm_status e = query_common(cfg, st, R, Q, qx, region, grid, &g);
    if (!e) e = bsdf_check(bsdf, Q);
    if (e) return e;
    if (Q > 0 && (!dir || !pdf_out)) return fail(SDMM_ERR_INVALID_ARG, "dir/pdf_out are NULL");
    if (Q == 0) return SDMM_OK;
    SDMM_CUDA(launch_product(stream, OP_PDF, pow2_ceil(cfg->K), query_grid(Q), st->qtab, cfg->K, R, Q, qx, region, g,
                             bsdf->w, bsdf->mu, bsdf->L, bsdf->J, 0, nullptr, dir, nullptr, pdf_out, nullptr),
              "product_pdf");
    return SDMM_OK;
}

sdmm_status sdmm_pdf(const sdmm_config* cfg, const sdmm_state* st, int64_t R, int64_t Q,
                     const float* qx, const int32_t* region, const sdmm_grid* grid, const float* dir,
                     float* pdf_out, sdmm_stream stream) {
    ProfileScope prof_("pdf", stream);
    GridF g;
    sdmm_status e = query_common(cfg, st, R, Q, qx, region, grid, &g);
    if (e) return e;
    if (Q > 0 && (!dir || !pdf_out)) return fail(SDMM_ERR_INVALID_ARG, "dir/pdf_out are NULL");
    if (Q == 0) return SDMM_OK;
    SDMM_CUDA(launch_query(stream, OP_PDF, pow2_ceil(cfg->K), query_grid(Q), st->qtab, cfg->K, R, Q, qx,
                           region, g, 0, nullptr, dir, nullptr, nullptr, nullptr, nullptr, pdf_out,
                           nullptr),
              "pdf");
    return SDMM_OK;
}

// ---------------------------------------------------------------- objective
static sdmm_status objective_common(const sdmm_config* cfg, const sdmm_samples* s,
                                    const double* prior_scale, const sdmm_state* st, double* F_out,
                                    const double* dF, float* gd, float* gL, float* ga, void* workspace,
                                    size_t ws_bytes, cudaStream_t stream) {
    sdmm_status e;
    if ((e = check_config(cfg)) || (e = check_samples(s)) || (e = check_state(st, false))) return e;
    if (!st->n_seen) return fail(SDMM_ERR_INVALID_ARG, "state.n_seen is NULL");
    if (cfg->prior_scale_mode == SDMM_PRIOR_SCALE_ARRAY && !prior_scale)
        return fail(SDMM_ERR_INVALID_ARG, "prior_scale_mode ARRAY needs prior_scale");
    const Layout L = layout(cfg, s->R, s->N, choose_chunk(cfg, s->N));
    if ((e = check_ws(workspace, ws_bytes, L))) return e;
    const int nsm = sm_count();
    if (nsm <= 0) return fail(SDMM_ERR_CUDA, "no CUDA device");
    const WsPtrs w = ws_ptrs(workspace, L);
    const int KP = pow2_ceil(cfg->K);
    // the specialised E-step's whitened statistics serve the adjoint too
    // (converted per component in the reduction); the generic kernel
    // accumulates the adjoint's own for K <= 2
    const int ystats = estep_fast_supported(KP);
    SDMM_CUDA(launch_set_desc(stream, w.hdr, make_desc(s, prior_scale, nullptr)), "set_desc");
    SDMM_CUDA(launch_build_chunks(stream, w.hdr, w.cb, w.cr, nullptr, L.chunk, 1, L.max_chunks), "build_chunks");
    SDMM_CUDA(launch_accumulate(stream, (dF && !ystats) ? MODE_GRAD : MODE_FIT, KP, nsm * default_ctas(cfg),
                                w.hdr, w.cb, w.cr, st->etab, cfg->K, L.chunk, cfg->estep_density, w.partial,
                                L.ps, 0, nullptr, cfg->dir_coords == SDMM_DIR_EUCLIDEAN, 1),
              "accumulate");
    SDMM_CUDA(launch_reduce_objective(stream, s->R, w.hdr, w.cb, w.partial, L.ps, *cfg, *st, F_out, dF,
                                      gd, gL, ga, ystats),
              "reduce_objective");
    return SDMM_OK;
}

sdmm_status sdmm_objective(const sdmm_config* cfg, const sdmm_samples* s, const double* prior_scale,
                           const sdmm_state* st, double* F_out, void* workspace, size_t ws_bytes,
                           sdmm_stream stream) {
    ProfileScope prof_("objective", stream);
    if (!F_out) return fail(SDMM_ERR_INVALID_ARG, "F_out is NULL");
    return objective_common(cfg, s, prior_scale, st, F_out, nullptr, nullptr, nullptr, nullptr,
                            workspace, ws_bytes, stream);
}

sdmm_status sdmm_objective_backward(const sdmm_config* cfg, const sdmm_samples* s,
                                    const double* prior_scale, const sdmm_state* st, const double* dF,
                                    float* g_delta, float* g_L, float* g_logit, void* workspace,
                                    size_t ws_bytes, sdmm_stream stream) {
    ProfileScope prof_("objective_backward", stream);
    if (!dF || !g_delta || !g_L || !g_logit) return fail(SDMM_ERR_INVALID_ARG, "dF/gradient outputs are NULL");
    return objective_common(cfg, s, prior_scale, st, nullptr, dF, g_delta, g_L, g_logit, workspace,
                            ws_bytes, stream);
}

// ---------------------------------------------------------------- plans
struct sdmm_fit_plan {
    FitLaunch f;
    int64_t N_max;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    std::vector<cudaEvent_t> cap_events;       // events recorded by the graph's event nodes
    std::vector<cudaGraphNode_t> ev_nodes;     // node of cap_events[i]
    std::vector<cudaEvent_t> pool;             // timing: 2*iters events per run
    int32_t capacity = 0;
    int32_t runs = 0;
    // batches from host memory: two staging slots, copies on their own stream
    cudaStream_t copy = nullptr;
    cudaEvent_t ready[2] = {nullptr, nullptr};  // slot's copy done (copy stream)
    cudaEvent_t freed[2] = {nullptr, nullptr};  // slot's replay done (caller's stream)
    int64_t host_runs = 0;
};

static size_t align256(size_t b) { return (b + 255) & ~(size_t)255; }
static size_t staging_slot_bytes(const sdmm_fit_plan* p) {
    return 7 * align256((size_t)p->N_max * sizeof(float)) + align256((size_t)(p->f.R + 1) * sizeof(int64_t));
}

sdmm_status sdmm_fit_plan_create(const sdmm_config* cfg, int64_t R, int64_t N_max, int32_t iters,
                                 sdmm_state* st, void* workspace, size_t ws_bytes, sdmm_stream stream,
                                 sdmm_fit_plan** plan_out) {
    sdmm_status e;
    if ((e = check_config(cfg)) || (e = check_state(st, true))) return e;
    if (!plan_out) return fail(SDMM_ERR_INVALID_ARG, "plan_out is NULL");
    *plan_out = nullptr;
    if (R < 1 || N_max < 0 || iters < 1) return fail(SDMM_ERR_INVALID_ARG, "R, N_max, iters out of range");
    const Layout L = layout(cfg, R, N_max, choose_chunk(cfg, N_max));
    if ((e = check_ws(workspace, ws_bytes, L))) return e;
    const int nsm = sm_count();
    if (nsm <= 0) return fail(SDMM_ERR_CUDA, "no CUDA device");
    sdmm_fit_plan* p = new sdmm_fit_plan();
    p->f = FitLaunch{*cfg, *st, L, ws_ptrs(workspace, L), R, iters, nsm * default_ctas(cfg), 1};
    p->N_max = N_max;
    p->cap_events.resize(2 * iters);
    for (auto& ev : p->cap_events) {
        if (cudaEventCreate(&ev) != cudaSuccess) {
            sdmm_fit_plan_destroy(p);
            return fail(SDMM_ERR_CUDA, "cudaEventCreate failed");
        }
    }
    cudaStream_t cs;
    if (cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking) != cudaSuccess) {
        sdmm_fit_plan_destroy(p);
        return fail(SDMM_ERR_CUDA, "cudaStreamCreate failed");
    }
    (void)stream;
    cudaError_t ce = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
    sdmm_status se = SDMM_OK;
    if (ce == cudaSuccess) {
        se = enqueue_fit(p->f, cs, &p->cap_events);
        ce = cudaStreamEndCapture(cs, &p->graph);
    }
    cudaStreamDestroy(cs);
    if (se != SDMM_OK || ce != cudaSuccess) {
        sdmm_fit_plan_destroy(p);
        return se != SDMM_OK ? se : cuda_fail(ce, "graph capture");
    }
    // locate the event-record nodes so that each run can retarget them
    size_t n = 0;
    cudaGraphGetNodes(p->graph, nullptr, &n);
    std::vector<cudaGraphNode_t> nodes(n);
    cudaGraphGetNodes(p->graph, nodes.data(), &n);
    p->ev_nodes.assign(p->cap_events.size(), nullptr);
    for (auto nd : nodes) {
        cudaGraphNodeType t;
        cudaGraphNodeGetType(nd, &t);
        if (t != cudaGraphNodeTypeEventRecord) continue;
        cudaEvent_t ev;
        cudaGraphEventRecordNodeGetEvent(nd, &ev);
        for (size_t i = 0; i < p->cap_events.size(); ++i)
            if (p->cap_events[i] == ev) p->ev_nodes[i] = nd;
    }
    ce = cudaGraphInstantiate(&p->exec, p->graph, 0);
    if (ce != cudaSuccess) {
        sdmm_fit_plan_destroy(p);
        return cuda_fail(ce, "graph instantiate");
    }
    *plan_out = p;
    return SDMM_OK;
}

sdmm_status sdmm_fit_plan_run(sdmm_fit_plan* p, const sdmm_samples* s, const double* prior_scale,
                              float* loglik_out, sdmm_stream stream) {
    ProfileScope prof_("fit_plan_run", stream);
    sdmm_status e;
    if (!p) return fail(SDMM_ERR_INVALID_ARG, "plan is NULL");
    if ((e = check_samples(s))) return e;
    if (s->R != p->f.R) return fail(SDMM_ERR_INVALID_ARG, "batch R %lld != plan R %lld", (long long)s->R, (long long)p->f.R);
    if (s->N > p->N_max) return fail(SDMM_ERR_INVALID_ARG, "batch N %lld > plan N_max %lld", (long long)s->N, (long long)p->N_max);
    if (p->f.cfg.prior_scale_mode == SDMM_PRIOR_SCALE_ARRAY && !prior_scale)
        return fail(SDMM_ERR_INVALID_ARG, "prior_scale_mode ARRAY needs prior_scale");
    if (p->capacity > 0 && p->runs < p->capacity) {
        for (size_t i = 0; i < p->ev_nodes.size(); ++i) {
            if (!p->ev_nodes[i]) continue;
            SDMM_CUDA(cudaGraphExecEventRecordNodeSetEvent(p->exec, p->ev_nodes[i],
                                                           p->pool[(size_t)p->runs * p->ev_nodes.size() + i]),
                      "retarget event");
        }
    }
    SDMM_CUDA(launch_set_desc(stream, p->f.w.hdr, make_desc(s, prior_scale, loglik_out)), "set_desc");
    SDMM_CUDA(cudaGraphLaunch(p->exec, stream), "graph launch");
    if (p->capacity > 0 && p->runs < p->capacity) ++p->runs;
    return SDMM_OK;
}

sdmm_status sdmm_fit_plan_staging_size(const sdmm_fit_plan* p, size_t* bytes_out) {
    if (!p || !bytes_out) return fail(SDMM_ERR_INVALID_ARG, "plan or bytes_out is NULL");
    *bytes_out = 2 * staging_slot_bytes(p);
    return SDMM_OK;
}

static bool on_device(const void* ptr) {
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, ptr) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeDevice;
}

sdmm_status sdmm_fit_plan_run_host(sdmm_fit_plan* p, const sdmm_samples* hs, void* staging, size_t staging_bytes,
                                   const double* prior_scale, float* loglik_out, sdmm_stream stream) {
    ProfileScope prof_("fit_plan_run_host", stream);
    sdmm_status e;
    if (!p) return fail(SDMM_ERR_INVALID_ARG, "plan is NULL");
    if ((e = check_samples(hs))) return e;
    if (hs->R != p->f.R) return fail(SDMM_ERR_INVALID_ARG, "batch R %lld != plan R %lld", (long long)hs->R, (long long)p->f.R);
    if (hs->N > p->N_max) return fail(SDMM_ERR_INVALID_ARG, "batch N %lld > plan N_max %lld", (long long)hs->N, (long long)p->N_max);
    const size_t slot_bytes = staging_slot_bytes(p);
    if (!staging || (reinterpret_cast<uintptr_t>(staging) & 255u) || staging_bytes < 2 * slot_bytes)
        return fail(SDMM_ERR_WORKSPACE, "staging must be 256-byte aligned device memory of %zu bytes", 2 * slot_bytes);
    if (on_device(hs->offsets) || (hs->N > 0 && on_device(hs->px)))
        return fail(SDMM_ERR_INVALID_ARG, "sdmm_fit_plan_run_host takes a batch in host memory");
    if (!p->copy) {
        SDMM_CUDA(cudaStreamCreateWithFlags(&p->copy, cudaStreamNonBlocking), "copy stream");
        for (int i = 0; i < 2; ++i) {
            SDMM_CUDA(cudaEventCreateWithFlags(&p->ready[i], cudaEventDisableTiming), "event");
            SDMM_CUDA(cudaEventCreateWithFlags(&p->freed[i], cudaEventDisableTiming), "event");
        }
    }
    const int slot = (int)(p->host_runs & 1);
    char* base = static_cast<char*>(staging) + (size_t)slot * slot_bytes;
    const size_t col = align256((size_t)p->N_max * sizeof(float));
    // the slot is rewritten once the replay that last read it is done; a fresh
    // slot waits for the work already queued on the caller's stream
    if (p->host_runs < 2) SDMM_CUDA(cudaEventRecord(p->freed[slot], stream), "event record");
    SDMM_CUDA(cudaStreamWaitEvent(p->copy, p->freed[slot], 0), "wait");
    const float* src[7] = {hs->px, hs->py, hs->pz, hs->ox, hs->oy, hs->oz, hs->w};
    float* dst[7];
    for (int i = 0; i < 7; ++i) {
        dst[i] = reinterpret_cast<float*>(base + (size_t)i * col);
        if (hs->N > 0)
            SDMM_CUDA(cudaMemcpyAsync(dst[i], src[i], (size_t)hs->N * sizeof(float), cudaMemcpyHostToDevice, p->copy),
                      "H2D samples");
    }
    int64_t* doff = reinterpret_cast<int64_t*>(base + 7 * col);
    SDMM_CUDA(cudaMemcpyAsync(doff, hs->offsets, (size_t)(hs->R + 1) * sizeof(int64_t), cudaMemcpyHostToDevice,
                              p->copy),
              "H2D offsets");
    SDMM_CUDA(cudaEventRecord(p->ready[slot], p->copy), "event record");
    SDMM_CUDA(cudaStreamWaitEvent(stream, p->ready[slot], 0), "wait");
    const sdmm_samples ds = {dst[0], dst[1], dst[2], dst[3], dst[4], dst[5], dst[6], doff, hs->R, hs->N};
    if ((e = sdmm_fit_plan_run(p, &ds, prior_scale, loglik_out, stream))) return e;
    SDMM_CUDA(cudaEventRecord(p->freed[slot], stream), "event record");
    ++p->host_runs;
    return SDMM_OK;
}

sdmm_status sdmm_fit_plan_enable_timing(sdmm_fit_plan* p, int32_t capacity) {
    if (!p || capacity < 1) return fail(SDMM_ERR_INVALID_ARG, "plan NULL or capacity < 1");
    for (auto ev : p->pool) cudaEventDestroy(ev);
    p->pool.assign((size_t)capacity * p->ev_nodes.size(), nullptr);
    for (auto& ev : p->pool) SDMM_CUDA(cudaEventCreate(&ev), "cudaEventCreate");
    p->capacity = capacity;
    p->runs = 0;
    return SDMM_OK;
}

sdmm_status sdmm_fit_plan_timing(sdmm_fit_plan* p, float* ms_out, int32_t max, int32_t* n_out) {
    if (!p || !n_out || (max > 0 && !ms_out)) return fail(SDMM_ERR_INVALID_ARG, "bad arguments");
    const size_t per = p->ev_nodes.size();
    int32_t n = 0;
    for (int32_t r = 0; r < p->runs; ++r)
        for (size_t i = 0; i + 1 < per; i += 2) {
            cudaEvent_t a = p->pool[(size_t)r * per + i], b = p->pool[(size_t)r * per + i + 1];
            SDMM_CUDA(cudaEventSynchronize(b), "event sync");
            float ms = 0.f;
            SDMM_CUDA(cudaEventElapsedTime(&ms, a, b), "event elapsed");
            if (n < max) ms_out[n] = ms;
            ++n;
        }
    *n_out = std::min(n, max);
    p->runs = 0;
    return SDMM_OK;
}

sdmm_status sdmm_fit_plan_destroy(sdmm_fit_plan* p) {
    if (!p) return SDMM_OK;
    if (p->exec) cudaGraphExecDestroy(p->exec);
    if (p->graph) cudaGraphDestroy(p->graph);
    for (auto ev : p->cap_events)
        if (ev) cudaEventDestroy(ev);
    for (auto ev : p->pool)
        if (ev) cudaEventDestroy(ev);
    for (int i = 0; i < 2; ++i) {
        if (p->ready[i]) cudaEventDestroy(p->ready[i]);
        if (p->freed[i]) cudaEventDestroy(p->freed[i]);
    }
    if (p->copy) cudaStreamDestroy(p->copy);
    delete p;
    return SDMM_OK;
}

// ---------------------------------------------------------------- tensor-core self-test
sdmm_status sdmm_tc_selftest(int32_t kind, int32_t N, int32_t Kd, const float* A, const float* B, float* D,
                             int32_t variant, int32_t* status, sdmm_stream stream) {
    if (kind != 0 && kind != 1) return fail(SDMM_ERR_INVALID_ARG, "kind %d: 0 (BF16) or 1 (TF32)", kind);
    if (N < 16 || N > 256 || N % 16) return fail(SDMM_ERR_INVALID_ARG, "N = %d: multiple of 16 in [16, 256]", N);
    const int kq = kind == 0 ? 16 : 8;
    if (Kd < kq || Kd > 64 || Kd % kq) return fail(SDMM_ERR_INVALID_ARG, "Kd = %d: multiple of %d, at most 64", Kd, kq);
    if (variant < 0 || variant > 31) return fail(SDMM_ERR_INVALID_ARG, "variant %d", variant);
    if (kind != 0 && (variant & 6)) return fail(SDMM_ERR_INVALID_ARG, "MN-major operands are tested for BF16 only");
    if (!A || !B || !D || !status) return fail(SDMM_ERR_INVALID_ARG, "NULL pointer");
    SDMM_CUDA(launch_tc_selftest(stream, kind, N, Kd, A, B, D, variant, status), "tc_selftest");
    return SDMM_OK;
}

sdmm_status sdmm_validate_samples(const sdmm_samples* s, float unit_tol, int64_t* counts, sdmm_stream stream) {
    if (!s) return fail(SDMM_ERR_INVALID_ARG, "samples is NULL");
    if (s->N < 0) return fail(SDMM_ERR_INVALID_ARG, "N = %lld", (long long)s->N);
    if (s->N > 0 && (!s->px || !s->py || !s->pz || !s->ox || !s->oy || !s->oz || !s->w))
        return fail(SDMM_ERR_INVALID_ARG, "sample streams are NULL");
    if (!counts) return fail(SDMM_ERR_INVALID_ARG, "counts is NULL");
    if (!(unit_tol > 0.f) || !(unit_tol < 1.f)) return fail(SDMM_ERR_INVALID_ARG, "unit_tol must be in (0, 1)");
    ProfileScope prof_("validate_samples", stream);
    BatchDesc d{};
    d.p[0] = s->px; d.p[1] = s->py; d.p[2] = s->pz; d.p[3] = s->ox; d.p[4] = s->oy; d.p[5] = s->oz; d.p[6] = s->w;
    SDMM_CUDA(launch_validate(static_cast<cudaStream_t>(stream), d, s->N, unit_tol,
                              reinterpret_cast<unsigned long long*>(counts), std::max(1, sm_count()) * 4),
              "validate_samples");
    return SDMM_OK;
}

sdmm_status sdmm_wait_selftest(int64_t limit_ns, int32_t arrive, int32_t* status, int64_t* elapsed_ns,
                               sdmm_stream stream) {
    if (limit_ns < 1 || limit_ns > 2000000000ll) return fail(SDMM_ERR_INVALID_ARG, "limit_ns %lld: 1 .. 2e9", (long long)limit_ns);
    if (!status || !elapsed_ns) return fail(SDMM_ERR_INVALID_ARG, "NULL pointer");
    SDMM_CUDA(launch_wait_selftest(stream, (uint64_t)limit_ns, arrive != 0, status,
                                   reinterpret_cast<unsigned long long*>(elapsed_ns)),
              "wait_selftest");
    return SDMM_OK;
}

// ---------------------------------------------------------------- fixed scratch
sdmm_status sdmm_fit_regions_noalloc(const sdmm_config* cfg, const sdmm_samples* s, int32_t iters,
                                     const double* prior_scale, sdmm_state* st, float* loglik_out,
                                     sdmm_stream stream) {
    ProfileScope prof_("fit_regions_noalloc", stream);
    sdmm_status e;
    if ((e = check_config(cfg)) || (e = check_samples(s)) || (e = check_state(st, true))) return e;
    if (iters < 1) return fail(SDMM_ERR_INVALID_ARG, "iters = %d must be >= 1", iters);
    if (cfg->prior_scale_mode == SDMM_PRIOR_SCALE_ARRAY && !prior_scale)
        return fail(SDMM_ERR_INVALID_ARG, "prior_scale_mode ARRAY needs prior_scale");
    const Layout L = layout(cfg, s->R, s->N, choose_chunk(cfg, s->N));
    if (L.total > (size_t)SDMM_NOALLOC_SCRATCH_BYTES)
        return fail(SDMM_ERR_WORKSPACE,
                    "sdmm_fit_regions_noalloc: this problem (R = %lld, N = %lld, K = %d) needs %zu bytes "
                    "of scratch but the fixed scratch holds %zu; use sdmm_fit_regions with a workspace",
                    (long long)s->R, (long long)s->N, cfg->K, L.total, (size_t)SDMM_NOALLOC_SCRATCH_BYTES);
    void* ws = nullptr;
    if ((e = noalloc_scratch(&ws))) return e;
    const int nsm = sm_count();
    if (nsm <= 0) return fail(SDMM_ERR_CUDA, "no CUDA device");
    FitLaunch f{*cfg, *st, L, ws_ptrs(ws, L), s->R, iters, nsm * default_ctas(cfg), loglik_out != nullptr};
    SDMM_CUDA(launch_set_desc(stream, f.w.hdr, make_desc(s, prior_scale, loglik_out)), "set_desc");
    return enqueue_fit(f, stream, nullptr);
}

// ---------------------------------------------------------------- autotuner
sdmm_status sdmm_autotune(const sdmm_config* cfg, const sdmm_samples* s, const sdmm_state* st,
                          void* workspace, size_t ws_bytes, sdmm_stream stream, int32_t* chunk_out,
                          int32_t* ctas_out, float* best_ms_out) {
    sdmm_status e;
    if ((e = check_config(cfg)) || (e = check_samples(s)) || (e = check_state(st, false))) return e;
    if (!chunk_out || !ctas_out) return fail(SDMM_ERR_INVALID_ARG, "outputs are NULL");
    const int nsm = sm_count();
    if (nsm <= 0) return fail(SDMM_ERR_CUDA, "no CUDA device");
    const int KP = pow2_ceil(cfg->K);
    cudaEvent_t a, b;
    SDMM_CUDA(cudaEventCreate(&a), "event");
    SDMM_CUDA(cudaEventCreate(&b), "event");
    float best = INFINITY;
    int best_c = 0, best_g = 0;
    const int chunks[] = {256, 512, 1024, 2048, 4096, 8192};
    // the specialised E-step sizes its own grid: only the chunk is tuned
    const int g_max = estep_fast_supported(KP) ? 1 : 4;
    for (int c : chunks) {
        const Layout L = layout(cfg, s->R, s->N, c);
        if (L.total > ws_bytes || !workspace) continue;
        const WsPtrs w = ws_ptrs(workspace, L);
        for (int g = 1; g <= g_max; ++g) {
            float tmin = INFINITY;
            for (int rep = 0; rep < 4; ++rep) {
                if (launch_set_desc(stream, w.hdr, make_desc(s, nullptr, nullptr)) != cudaSuccess ||
                    launch_build_chunks(stream, w.hdr, w.cb, w.cr, nullptr, c, cfg->min_samples, L.max_chunks) != cudaSuccess)
                    return fail(SDMM_ERR_CUDA, "autotune launch");
                cudaEventRecord(a, stream);
                if (launch_accumulate(stream, MODE_FIT, KP, nsm * g, w.hdr, w.cb, w.cr, st->etab, cfg->K, c,
                                      cfg->estep_density, w.partial, L.ps, 0, nullptr,
                                      cfg->dir_coords == SDMM_DIR_EUCLIDEAN) != cudaSuccess)
                    return fail(SDMM_ERR_CUDA, "autotune launch");
                cudaEventRecord(b, stream);
                SDMM_CUDA(cudaEventSynchronize(b), "autotune sync");
                float ms = 0.f;
                cudaEventElapsedTime(&ms, a, b);
                if (rep > 0) tmin = std::min(tmin, ms);
            }
            if (tmin < best) {
                best = tmin;
                best_c = c;
                best_g = g;
            }
        }
    }
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    if (best_c == 0) return fail(SDMM_ERR_WORKSPACE, "workspace too small for any candidate");
    *chunk_out = best_c;
    *ctas_out = g_max == 1 ? 0 : best_g;
    if (best_ms_out) *best_ms_out = best;
    return SDMM_OK;
}


// ===========================================================================
// Spatial kD-tree (Sec. 4.2, Sec. 4.3)
}  // extern "C"

namespace {

struct KdLayout {
    size_t rec[2], seg_off[2], seg_node[2], seg_parent[2], seg_axis, seg_split, seg_split_f, split_f, seg_flag, seg_new, seg_sum,
        seg_left, tile_seg, tile_start, tile_left, tile_prefix, seg_tile0, counters, rx_hist, rx_bsum, total;
    int64_t max_tiles;
};

KdLayout kd_layout(const sdmm_kdtree* t, int64_t N) {
    KdLayout L{};
    const size_t S = (size_t)t->cap_leaves + 1;
    L.max_tiles = N / kKdTile + (int64_t)t->cap_leaves + 1;
    const size_t T = (size_t)L.max_tiles;
    size_t o = 0;
    auto take = [&](size_t bytes) {
        const size_t at = o;
        o = align_up(o + bytes);
        return at;
    };
    for (int b = 0; b < 2; ++b) {
        L.rec[b] = take(sizeof(float4) * (size_t)N);
        L.seg_off[b] = take(sizeof(int64_t) * (S + 1));
        L.seg_node[b] = take(sizeof(int32_t) * S);
        L.seg_parent[b] = take(sizeof(int64_t) * S);
    }
    L.seg_axis = take(sizeof(int32_t) * S);
    L.seg_split = take(sizeof(double) * S);
    L.seg_split_f = take(sizeof(float) * S);
    L.split_f = take(sizeof(float) * (size_t)t->cap_nodes);
    L.seg_flag = take(sizeof(int32_t) * S);
    L.seg_new = take(sizeof(int32_t) * S);
    L.seg_sum = take(sizeof(unsigned long long) * 6 * S);
    L.seg_left = take(sizeof(unsigned long long) * S);
    L.tile_seg = take(sizeof(int32_t) * T);
    L.tile_start = take(sizeof(int64_t) * T);
    L.tile_left = take(sizeof(int32_t) * T);
    L.tile_prefix = take(sizeof(int64_t) * T);
    L.seg_tile0 = take(sizeof(int32_t) * (S + 1));
    L.counters = take(sizeof(int32_t) * 4);
    L.rx_hist = take(sizeof(uint32_t) * (size_t)rx_hist_entries(N));
    L.rx_bsum = take(sizeof(uint32_t) * ((size_t)rx_scan_blocks(N) + 1));
    L.total = o;
    return L;
}

KdWork kd_work(void* ws, const KdLayout& L) {
    char* b = static_cast<char*>(ws);
    KdWork w{};
    for (int i = 0; i < 2; ++i) {
        w.rec[i] = reinterpret_cast<float4*>(b + L.rec[i]);
        w.seg_off[i] = reinterpret_cast<int64_t*>(b + L.seg_off[i]);
        w.seg_node[i] = reinterpret_cast<int32_t*>(b + L.seg_node[i]);
        w.seg_parent[i] = reinterpret_cast<int64_t*>(b + L.seg_parent[i]);
    }
    w.seg_axis = reinterpret_cast<int32_t*>(b + L.seg_axis);
    w.seg_split = reinterpret_cast<double*>(b + L.seg_split);
    w.seg_split_f = reinterpret_cast<float*>(b + L.seg_split_f);
    w.split_f = reinterpret_cast<float*>(b + L.split_f);
    w.seg_flag = reinterpret_cast<int32_t*>(b + L.seg_flag);
    w.seg_new = reinterpret_cast<int32_t*>(b + L.seg_new);
    w.seg_sum = reinterpret_cast<unsigned long long*>(b + L.seg_sum);
    w.seg_left = reinterpret_cast<unsigned long long*>(b + L.seg_left);
    w.tile_seg = reinterpret_cast<int32_t*>(b + L.tile_seg);
    w.tile_start = reinterpret_cast<int64_t*>(b + L.tile_start);
    w.tile_left = reinterpret_cast<int32_t*>(b + L.tile_left);
    w.tile_prefix = reinterpret_cast<int64_t*>(b + L.tile_prefix);
    w.seg_tile0 = reinterpret_cast<int32_t*>(b + L.seg_tile0);
    w.counters = reinterpret_cast<int32_t*>(b + L.counters);
    w.rx_hist = reinterpret_cast<uint32_t*>(b + L.rx_hist);
    w.rx_bsum = reinterpret_cast<uint32_t*>(b + L.rx_bsum);
    w.max_tiles = L.max_tiles;
    return w;
}

sdmm_status kd_check(const sdmm_kdtree* t) {
    if (!t || !t->axis || !t->split || !t->left || !t->leaf) return fail(SDMM_ERR_INVALID_ARG, "kD-tree arrays are NULL");
    if (t->n_nodes < 1 || t->n_nodes > t->cap_nodes || t->n_leaves < 1 || t->n_leaves > t->cap_leaves)
        return fail(SDMM_ERR_INVALID_ARG, "kD-tree counts %d nodes / %d leaves exceed capacities %d / %d",
                    t->n_nodes, t->n_leaves, t->cap_nodes, t->cap_leaves);
    return SDMM_OK;
}

sdmm_status kd_streams(const sdmm_samples* in, const sdmm_sample_buffers* out) {
    if (!in || !out) return fail(SDMM_ERR_INVALID_ARG, "samples are NULL");
    if (in->N < 0 || in->N >= (int64_t(1) << 31)) return fail(SDMM_ERR_INVALID_ARG, "N = %lld: 0 <= N < 2^31", (long long)in->N);
    if (in->N > 0 && (!in->px || !in->py || !in->pz || !in->ox || !in->oy || !in->oz || !in->w))
        return fail(SDMM_ERR_INVALID_ARG, "input streams are NULL");
    if (!out->px || !out->py || !out->pz || !out->ox || !out->oy || !out->oz || !out->w || !out->offsets)
        return fail(SDMM_ERR_INVALID_ARG, "output streams are NULL");
    return SDMM_OK;
}

BatchDesc desc_of(const sdmm_samples* s) {
    BatchDesc d{};
    d.p[0] = s->px; d.p[1] = s->py; d.p[2] = s->pz; d.p[3] = s->ox; d.p[4] = s->oy; d.p[5] = s->oz; d.p[6] = s->w;
    return d;
}

BatchDesc desc_of(const sdmm_sample_buffers* s) {
    BatchDesc d{};
    d.p[0] = s->px; d.p[1] = s->py; d.p[2] = s->pz; d.p[3] = s->ox; d.p[4] = s->oy; d.p[5] = s->oz; d.p[6] = s->w;
    return d;
}

}  // namespace

extern "C" {

sdmm_status sdmm_kdtree_grid(sdmm_kdtree* t, int32_t levels, sdmm_stream stream) {
    if (!t || !t->axis || !t->split || !t->left || !t->leaf) return fail(SDMM_ERR_INVALID_ARG, "kD-tree arrays are NULL");
    if (levels < 0 || levels > 7) return fail(SDMM_ERR_INVALID_ARG, "levels %d: 0..7", levels);
    const int64_t nodes = (int64_t(1) << (3 * levels + 1)) - 1, leaves = int64_t(1) << (3 * levels);
    if (nodes > t->cap_nodes || leaves > t->cap_leaves)
        return fail(SDMM_ERR_WORKSPACE, "grid of %lld nodes / %lld leaves exceeds capacities %d / %d",
                    (long long)nodes, (long long)leaves, t->cap_nodes, t->cap_leaves);
    SDMM_CUDA(launch_kd_grid(stream, levels, t->axis, t->split, t->left, t->leaf), "kd_grid");
    SDMM_CUDA(cudaStreamSynchronize(stream), "kd_grid");
    t->n_nodes = (int32_t)nodes;
    t->n_leaves = (int32_t)leaves;
    return SDMM_OK;
}

sdmm_status sdmm_kdtree_lookup(const sdmm_kdtree* t, int64_t Q, const float* px, const float* py, const float* pz,
                               int32_t* leaf, sdmm_stream stream) {
    sdmm_status e = kd_check(t);
    if (e) return e;
    if (Q < 0) return fail(SDMM_ERR_INVALID_ARG, "Q < 0");
    if (Q > 0 && (!px || !py || !pz || !leaf)) return fail(SDMM_ERR_INVALID_ARG, "points/leaf are NULL");
    SDMM_CUDA(launch_kd_lookup(stream, t->axis, t->split, t->left, t->leaf, t->n_nodes, Q, px, py, pz, leaf),
              "kd_lookup");
    return SDMM_OK;
}

sdmm_status sdmm_kdtree_workspace_size(const sdmm_kdtree* t, int64_t N, size_t* bytes) {
    if (!t || !bytes) return fail(SDMM_ERR_INVALID_ARG, "NULL argument");
    if (N < 0 || N >= (int64_t(1) << 31)) return fail(SDMM_ERR_INVALID_ARG, "N = %lld: 0 <= N < 2^31", (long long)N);
    if (t->cap_leaves < 1 || t->cap_nodes < 1) return fail(SDMM_ERR_INVALID_ARG, "capacities must be positive");
    *bytes = kd_layout(t, N).total;
    return SDMM_OK;
}

static sdmm_status kd_run(sdmm_kdtree* t, int binning, int64_t c, const sdmm_samples* in, sdmm_sample_buffers* out,
                          int64_t* leaf_parent, void* ws, size_t ws_bytes, sdmm_stream stream) {
    const KdLayout L = kd_layout(t, in->N);
    if (!ws) return fail(SDMM_ERR_INVALID_ARG, "workspace is NULL");
    if (reinterpret_cast<uintptr_t>(ws) % kAlign) return fail(SDMM_ERR_INVALID_ARG, "workspace must be 256-byte aligned");
    if (ws_bytes < L.total) return fail(SDMM_ERR_WORKSPACE, "workspace %zu bytes < required %zu", ws_bytes, L.total);
    const KdWork w = kd_work(ws, L);
    const int64_t N = in->N;
    if (binning) {
        // every sample's leaf, a stable radix sort by leaf, the gather and the offsets
        SDMM_CUDA(launch_kd_bin(stream, w, t->axis, t->split, t->left, t->leaf, t->n_nodes, t->n_leaves, N, in->px,
                                in->py, in->pz, desc_of(in), desc_of(out), out->offsets),
                  "kd_bin");
        SDMM_CUDA(cudaStreamSynchronize(stream), "kd_bin");
        out->R = t->n_leaves;
        out->N = N;
        return SDMM_OK;
    }
    const int32_t S0 = t->n_leaves;
    SDMM_CUDA(launch_kd_prepare(stream, w, t->axis, t->leaf, t->n_nodes, S0, in->offsets, N, in->px, in->py,
                                in->pz),
              "kd_prepare");
    const float4* rec = nullptr;
    int32_t S = 0;
    int64_t *seg_off = nullptr, *seg_parent = nullptr;
    int overflow = 0;
    int32_t n_nodes = t->n_nodes, n_leaves = t->n_leaves;
    SDMM_CUDA(kd_rounds(stream, w, c, t->axis, t->split, t->left, t->leaf, &n_nodes, &n_leaves,
                        t->cap_nodes, t->cap_leaves, S0, N, &rec, &seg_off, &seg_parent,
                        &S, &overflow),
              "kd_rounds");
    t->n_nodes = n_nodes;
    t->n_leaves = n_leaves;
    if (overflow)
        return fail(SDMM_ERR_WORKSPACE, "kD-tree capacities (%d nodes, %d leaves) too small", t->cap_nodes,
                    t->cap_leaves);
    SDMM_CUDA(launch_kd_gather(stream, N, rec, desc_of(in), desc_of(out)), "kd_gather");
    SDMM_CUDA(cudaMemcpyAsync(out->offsets, seg_off, sizeof(int64_t) * ((size_t)S + 1), cudaMemcpyDeviceToDevice,
                              stream),
              "kd_offsets");
    if (leaf_parent)
        SDMM_CUDA(cudaMemcpyAsync(leaf_parent, seg_parent, sizeof(int64_t) * (size_t)S, cudaMemcpyDeviceToDevice,
                                  stream),
                  "kd_parent");
    SDMM_CUDA(cudaStreamSynchronize(stream), "kd_run");
    out->R = S;
    out->N = N;
    return SDMM_OK;
}

sdmm_status sdmm_kdtree_bin(const sdmm_kdtree* t, const sdmm_samples* in, sdmm_sample_buffers* out, void* ws,
                            size_t ws_bytes, sdmm_stream stream) {
    ProfileScope prof_("kdtree_bin", stream);
    sdmm_status e = kd_check(t);
    if (!e) e = kd_streams(in, out);
    if (e) return e;
    // the tree is not modified by binning
    sdmm_kdtree tt = *t;
    return kd_run(&tt, 1, -1, in, out, nullptr, ws, ws_bytes, stream);
}

sdmm_status sdmm_kdtree_refine(sdmm_kdtree* t, int64_t c, const sdmm_samples* in, sdmm_sample_buffers* out,
                               int64_t* leaf_parent, void* ws, size_t ws_bytes, sdmm_stream stream) {
    ProfileScope prof_("kdtree_refine", stream);
    sdmm_status e = kd_check(t);
    if (!e) e = kd_streams(in, out);
    if (e) return e;
    if (c < 1) return fail(SDMM_ERR_INVALID_ARG, "c = %lld must be >= 1", (long long)c);
    if (!in->offsets || in->R != t->n_leaves)
        return fail(SDMM_ERR_INVALID_ARG, "in->R = %lld must equal the tree's %d leaves", (long long)in->R, t->n_leaves);
    if (!leaf_parent) return fail(SDMM_ERR_INVALID_ARG, "leaf_parent is NULL");
    return kd_run(t, 0, c, in, out, leaf_parent, ws, ws_bytes, stream);
}

sdmm_status sdmm_gather_regions(int32_t K, int64_t R_out, const int64_t* src, const sdmm_state* in,
                                sdmm_state* out, sdmm_stream stream) {
    if (K < 1 || K > SDMM_MAX_K) return fail(SDMM_ERR_INVALID_ARG, "K = %d", K);
    if (R_out < 0 || (R_out > 0 && (!src || !in || !out))) return fail(SDMM_ERR_INVALID_ARG, "NULL argument");
    if (R_out == 0) return SDMM_OK;
    SDMM_CUDA(launch_gather_state(stream, K, R_out, src, *in, *out), "gather_regions");
    return SDMM_OK;
}

}  // extern "C"
