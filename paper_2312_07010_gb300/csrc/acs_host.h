// acs_host.h -- host-side pieces shared by the translation units of libacs.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>
#include <string>
#include <vector>

#include "acs_kernels.cuh"

namespace acs {

// Adjoint recording state of a context (see acs_grad_bind in acs.h).
// A recorded CUDA graph of the adjoint unit: kind 0 = recording forward (a = first
// step, b = steps), kind 1 = backward sweep (a = recorded steps, b = checkpoint spacing).
struct GradGraph {
    int kind;
    int64_t a, b;
    cudaGraphExec_t exec;
};

struct GradState {
    bool active = false;
    char* buf = nullptr;
    size_t bytes = 0;
    int64_t max_steps = 0, every = 1;
    int64_t recorded = 0;  // steps recorded since the last set_state
    bool started = false;  // checkpoint 0 holds phi^0
    std::vector<GradGraph> graphs;
};

// Release the adjoint unit's recorded graphs (their kernels bake in pointers and
// coefficients, so any change of those invalidates them).
void grad_drop_graphs(GradState& G);

// What the other translation units may see of a context.
struct CtxView {
    int dims, bc, dtype;
    Geo g;
    size_t esize;
    double lam, dt, h, eps;
    void* phi;
    void* other;
    cudaStream_t stream;
    cudaStream_t cap;  // stream used for graph capture
    int* err;          // device flag set by kernels whose bounded waits gave up
    RedPartial* partials;
    double* result;
    int64_t steps_done;
    Coef<float> cf;
    Coef<double> cd;
    GradState* grad;
};

// Shape limit of every entry point: 1 <= n[k] and prod(n) <= 2^40 elements.  Each
// factor is checked against the limit divided by the product so far, before the
// multiplication, so no int64 product can wrap around.
constexpr int64_t kMaxElements = int64_t(1) << 40;
inline bool shape_ok(int dims, const int64_t* n) {
    int64_t total = 1;
    for (int k = 0; k < dims; ++k) {
        if (n[k] < 1 || n[k] > kMaxElements / total) return false;
        total *= n[k];
    }
    return true;
}

template <typename T>
Coef<T> make_coef(int dims, double lam, double dt, int scheme, bool mp_ok);
Geo make_geo(int dims, const int64_t* n);

// Kernel choice for ACS_KERNEL_AUTO (autotune cache, else a static rule).
void resolve_auto_kernel(int dims, int dtype, int bc, const Geo& g, int* kernel, int* depth);

// Implemented in acs_api.cu for the adjoint unit.
cudaError_t ctx_enqueue_steps(acs_ctx* c, int64_t n, cudaStream_t st);
cudaError_t ctx_launch_one(acs_ctx* c, const void* src, void* dst, cudaStream_t st);
CtxView ctx_view(acs_ctx* c);

// Implemented in acs_api.cu for the pipelined host-to-host runner (pipe.cu).
int ctx_enqueue_logged(acs_ctx* c, int64_t n_steps, int64_t every, double** d_log, int64_t* entries);
int ctx_check_err(acs_ctx* c);  // after a synchronization: ACS_E_TIMEOUT if a kernel gave up

// Tuning cache (tune_cache.cu): a text file of the autotuner's choices.
bool tune_cache_lookup(int dims, const int64_t* n, int bc, int dtype, int scheme, int* kernel, int* depth,
                       int* variant, int* chunk);
void tune_cache_store(int dims, const int64_t* n, int bc, int dtype, int scheme, int kernel, int depth, int variant,
                      int chunk, double us);
// The same for a workload class named by a string (the device is added to the key).
bool tune_cache_lookup_class(const std::string& cls, int* v4);
void tune_cache_store_class(const std::string& cls, const int* v4, double us);

// Implemented in adjoint.cu.
int grad_on_set_state(acs_ctx* c);
int grad_record_steps(acs_ctx* c, int64_t n);

}  // namespace acs
