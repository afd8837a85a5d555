// Host side of the learned variant selector: features, plan classes, the
// network's ABI entry points and the process-wide selector setting.
#include <cmath>
#include <cstring>
#include <mutex>

#include "kernels.cuh"
#include "planner.h"

namespace eiger {
eiger_status report_error(eiger_status s, const char* msg);

namespace {
std::mutex g_sel_mu;
const float* g_sel_params = nullptr;
float g_sel_mean[EIGER_MLP_IN];
float g_sel_scale[EIGER_MLP_IN];
}  // namespace

bool selector_get(const float** params, float* mean, float* scale) {
    std::lock_guard<std::mutex> lock(g_sel_mu);
    if (!g_sel_params) return false;
    *params = g_sel_params;
    std::memcpy(mean, g_sel_mean, sizeof g_sel_mean);
    std::memcpy(scale, g_sel_scale, sizeof g_sel_scale);
    return true;
}

void compute_features(const eiger_stats_t* b, const eiger_stats_t* ps, int64_t nb, int64_t np, int dtype,
                      size_t l2, float* f) {
    const double dnb = nb > 0 ? (double)nb : 1.0, dnp = np > 0 ? (double)np : 1.0;
    const bool have_b = b && b->n > 0;
    const double span = have_b ? (double)((uint64_t)b->max - (uint64_t)b->min) : 0.0;
    const bool narrow = have_b && (dtype == EIGER_I32 || (uint64_t)b->max - (uint64_t)b->min <= 0xFFFFFFFFull);
    const double ndv_b = have_b ? b->estimate : 0.0;
    const bool have_p = ps && ps->n > 0;
    const double ndv_p = have_p ? ps->estimate : 0.0;
    double overlap = 0.0;
    if (have_b && have_p) {
        const double lo = (double)(b->min > ps->min ? b->min : ps->min);
        const double hi = (double)(b->max < ps->max ? b->max : ps->max);
        const double width = (double)ps->max - (double)ps->min + 1.0;
        overlap = hi >= lo ? (hi - lo + 1.0) / width : 0.0;
        if (overlap > 1.0) overlap = 1.0;
    }
    const double slot = (dtype == EIGER_I32 || narrow) ? 8.0 : 16.0;
    const double table = (double)table_slots(nb, 0.5) * slot;
    f[0] = (float)std::log2(dnb);
    f[1] = (float)std::log2(dnp);
    f[2] = (float)std::log2(dnp / dnb);
    f[3] = dtype == EIGER_I32 ? 4.f : 8.f;
    f[4] = narrow ? 1.f : 0.f;
    f[5] = (float)std::log2(span + 1.0);
    f[6] = (float)std::log2(ndv_b + 1.0);
    f[7] = (float)(ndv_b / dnb);
    f[8] = (float)std::log2(ndv_p + 1.0);
    f[9] = have_p ? (float)(ndv_p / (double)ps->n) : 0.f;
    f[10] = (float)overlap;
    f[11] = (float)std::log2(table / (double)(l2 ? l2 : ((size_t)126 << 20)));
}

eiger_plan_t class_plan(int cls) {
    eiger_plan_t p{};
    p.load_factor = 0.5f;
    p.selector = 1;
    if (cls <= 0) {
        p.variant = EIGER_NPHJ;
    } else if (cls <= 5) {
        p.variant = EIGER_PHJ1;
        p.bits1 = 7 + cls;  // 8..12
    } else {
        const int B = 4 + cls;  // 10..18, split like the rules: pass 2 takes an odd count's extra bit
        p.variant = EIGER_PHJ2;
        p.bits1 = B / 2;
        p.bits2 = B - B / 2;
    }
    return p;
}

}  // namespace eiger

using namespace eiger;

extern "C" {

int32_t eiger_mlp_param_count(void) { return mlp_param_count(); }

eiger_status eiger_mlp_forward(const float* d_params, const float* d_x, int32_t n, float* d_logits, void* stream) {
    if (n < 0 || (n > 0 && (!d_params || !d_x || !d_logits)))
        return report_error(EIGER_ERR_INVALID_ARG, "bad network arguments");
    cudaError_t e = mlp_forward(d_params, d_x, n, d_logits, static_cast<cudaStream_t>(stream));
    return e == cudaSuccess ? EIGER_OK : report_error(EIGER_ERR_CUDA, cudaGetErrorString(e));
}

eiger_status eiger_mlp_grad_workspace(int32_t n, size_t* bytes) {
    if (n < 0 || !bytes) return report_error(EIGER_ERR_INVALID_ARG, "bad arguments");
    *bytes = mlp_grad_ws_bytes(n);
    return EIGER_OK;
}

eiger_status eiger_mlp_grad(const float* d_params, const float* d_x, const float* d_cost, int32_t n, float tau,
                            float* d_grad, float* d_loss, void* d_ws, size_t ws_bytes, void* stream) {
    if (n < 0 || (n > 0 && (!d_params || !d_x || !d_cost || !d_grad || !d_ws)))
        return report_error(EIGER_ERR_INVALID_ARG, "bad network arguments");
    if (!(tau >= 0.f)) return report_error(EIGER_ERR_INVALID_ARG, "tau must be >= 0");
    if (ws_bytes < mlp_grad_ws_bytes(n)) return report_error(EIGER_ERR_WORKSPACE, "workspace too small");
    cudaError_t e = mlp_grad(d_params, d_x, d_cost, n, tau, d_grad, d_loss, d_ws, static_cast<cudaStream_t>(stream));
    return e == cudaSuccess ? EIGER_OK : report_error(EIGER_ERR_CUDA, cudaGetErrorString(e));
}

eiger_status eiger_mlp_adam(float* d_params, const float* d_grad, float* d_m, float* d_v, int32_t step, float lr,
                            void* stream) {
    if (!d_params || !d_grad || !d_m || !d_v || step < 1 || !(lr > 0.f))
        return report_error(EIGER_ERR_INVALID_ARG, "bad optimiser arguments");
    cudaError_t e = mlp_adam(d_params, d_grad, d_m, d_v, step, lr, static_cast<cudaStream_t>(stream));
    return e == cudaSuccess ? EIGER_OK : report_error(EIGER_ERR_CUDA, cudaGetErrorString(e));
}

eiger_status eiger_features(const eiger_stats_t* build, const eiger_stats_t* probe_sample, int64_t nb, int64_t np,
                            eiger_dtype dtype, size_t l2_bytes, float out[EIGER_MLP_IN]) {
    if (!out || !build || nb < 0 || np < 0 || (dtype != EIGER_I32 && dtype != EIGER_I64))
        return report_error(EIGER_ERR_INVALID_ARG, "bad feature arguments");
    size_t l2 = l2_bytes;
    if (!l2) {
        DevInfo di;
        if (current_device_info(&di) == cudaSuccess && di.l2_bytes > 0)
            l2 = (size_t)di.l2_bytes;
        else
            cudaGetLastError();
    }
    compute_features(build, probe_sample, nb, np, dtype, l2, out);
    return EIGER_OK;
}

eiger_status eiger_class_plan(int32_t cls, eiger_plan_t* out) {
    if (!out || cls < 0 || cls >= EIGER_MLP_OUT) return report_error(EIGER_ERR_INVALID_ARG, "class outside 0..14");
    *out = class_plan(cls);
    return EIGER_OK;
}

eiger_status eiger_selector_set(const float* d_params, const float* h_mean, const float* h_scale) {
    std::lock_guard<std::mutex> lock(g_sel_mu);
    if (!d_params) {
        g_sel_params = nullptr;
        return EIGER_OK;
    }
    if (!h_mean || !h_scale) return report_error(EIGER_ERR_INVALID_ARG, "normalisation arrays are required");
    for (int i = 0; i < EIGER_MLP_IN; ++i)
        if (!(h_scale[i] > 0.f)) return report_error(EIGER_ERR_INVALID_ARG, "feature scales must be positive");
    std::memcpy(g_sel_mean, h_mean, sizeof g_sel_mean);
    std::memcpy(g_sel_scale, h_scale, sizeof g_sel_scale);
    g_sel_params = d_params;
    return EIGER_OK;
}

}  // extern "C"
