// pipe.cu -- pipelined host-to-host runs (acs_pipe_*): S contexts (slots) on one
// compute stream, each owning one device state, and two copy streams.  Job j uses
// slot j % S:
//   copy-in stream:  wait until the slot's previous job is copied out; H2D phi^0; mark
//   compute stream:  wait for the H2D; steps and logged reductions; mark
//   copy-out stream: wait for the compute; D2H phi^N and the log; mark
// so the copies of the neighbouring jobs overlap this job's steps.  With S = 2 the
// input copy of job j+1 follows the output copy of job j-1 within job j's compute;
// S = 3 lets the two copies run side by side and leaves a whole job of slack for a
// slow host link.  The steps are the contexts' own (graph replay of the tiled
// kernels), so results equal acs_run_logged's.
#include <cmath>
#include <new>
#include <vector>

#include "acs_host.h"

using namespace acs;

constexpr int kMaxSlots = 4;

struct acs_pipe {
    int slots = 0;
    acs_ctx* ctx[kMaxSlots] = {};
    size_t state_bytes = 0, work_bytes = 0;
    bool bound = false;
    cudaStream_t compute = nullptr, in = nullptr, out = nullptr;
    cudaEvent_t in_done[kMaxSlots] = {}, comp_done[kMaxSlots] = {}, out_done[kMaxSlots] = {};
    int next = 0;
    struct Pending {
        const double* log;
        int64_t entries;
    };
    std::vector<Pending> pending;
};

namespace {
constexpr size_t kPipeAlign = 256;
size_t pipe_align(size_t x) { return (x + kPipeAlign - 1) / kPipeAlign * kPipeAlign; }

void release_streams(acs_pipe* p) {
    for (int k = 0; k < kMaxSlots; ++k) {
        if (p->in_done[k]) cudaEventDestroy(p->in_done[k]);
        if (p->comp_done[k]) cudaEventDestroy(p->comp_done[k]);
        if (p->out_done[k]) cudaEventDestroy(p->out_done[k]);
        p->in_done[k] = p->comp_done[k] = p->out_done[k] = nullptr;
    }
    if (p->in) cudaStreamDestroy(p->in);
    if (p->out) cudaStreamDestroy(p->out);
    p->in = p->out = nullptr;
}
}  // namespace

extern "C" {

ACS_API int acs_pipe_create(int dims, const int64_t n[3], double eps, double dt, double h, int bc, int dtype,
                            int slots, acs_pipe** out) {
    if (!out || slots < 2 || slots > kMaxSlots) return ACS_E_INVAL;
    acs_pipe* p = new (std::nothrow) acs_pipe();
    if (!p) return ACS_E_NOMEM;
    p->slots = slots;
    int rc = ACS_OK;
    for (int k = 0; k < slots; ++k) {
        rc = acs_create(dims, n, eps, dt, h, bc, dtype, &p->ctx[k]);
        if (rc < 0) {
            acs_pipe_destroy(p);
            return rc;
        }
    }
    int64_t total = 1;
    for (int k = 0; k < dims; ++k) total *= n[k];
    p->state_bytes = pipe_align((size_t)total * (dtype == ACS_F32 ? 4 : 8));
    p->work_bytes = pipe_align(acs_work_bytes(p->ctx[0]));
    *out = p;
    return rc;
}

ACS_API size_t acs_pipe_bytes(const acs_pipe* p) { return p ? p->slots * (p->state_bytes + p->work_bytes) : 0; }

ACS_API int acs_pipe_bind(acs_pipe* p, void* d_buf, size_t bytes, void* stream) {
    if (!p || !d_buf || ((uintptr_t)d_buf % kPipeAlign)) return ACS_E_INVAL;
    if (bytes < acs_pipe_bytes(p)) return ACS_E_NOMEM;
    if (p->bound) {
        if (int rc = acs_pipe_wait(p); rc == ACS_E_CUDA) return rc;
    }
    release_streams(p);
    p->bound = false;
    p->compute = (cudaStream_t)stream;
    bool ok = cudaStreamCreateWithFlags(&p->in, cudaStreamNonBlocking) == cudaSuccess &&
              cudaStreamCreateWithFlags(&p->out, cudaStreamNonBlocking) == cudaSuccess;
    for (int k = 0; k < p->slots && ok; ++k)
        ok = cudaEventCreateWithFlags(&p->in_done[k], cudaEventDisableTiming) == cudaSuccess &&
             cudaEventCreateWithFlags(&p->comp_done[k], cudaEventDisableTiming) == cudaSuccess &&
             cudaEventCreateWithFlags(&p->out_done[k], cudaEventDisableTiming) == cudaSuccess;
    if (!ok) {
        release_streams(p);
        return ACS_E_CUDA;
    }
    char* base = (char*)d_buf;
    for (int k = 0; k < p->slots; ++k) {
        char* phi = base + k * (p->state_bytes + p->work_bytes);
        int rc = acs_bind(p->ctx[k], phi, phi + p->state_bytes, p->work_bytes, stream);
        if (rc) return rc;
    }
    p->next = 0;
    p->pending.clear();
    p->bound = true;
    return ACS_OK;
}

ACS_API acs_ctx* acs_pipe_context(acs_pipe* p, int slot) {
    if (!p || slot < 0 || slot >= p->slots) return nullptr;
    return p->ctx[slot];
}

ACS_API int acs_pipe_submit(acs_pipe* p, const void* h_in, void* h_out, int64_t n_steps, int64_t every,
                            double* h_log) {
    if (!p || !h_in || !h_out || n_steps < 0 || every < 0) return ACS_E_INVAL;
    if (every > 0 && (!h_log || n_steps / every + 1 > 4096)) return ACS_E_INVAL;
    if (!p->bound) return ACS_E_STATE;
    const int k = p->next;
    acs_ctx* c = p->ctx[k];
    const CtxView v = ctx_view(c);
    const size_t sb = (size_t)v.g.total * v.esize;
    // the slot's previous job has been copied out, so its state and log are free
    if (cudaStreamWaitEvent(p->in, p->out_done[k], 0) != cudaSuccess) return ACS_E_CUDA;
    if (cudaMemcpyAsync(v.phi, h_in, sb, cudaMemcpyHostToDevice, p->in) != cudaSuccess) return ACS_E_CUDA;
    if (cudaEventRecord(p->in_done[k], p->in) != cudaSuccess) return ACS_E_CUDA;
    if (cudaStreamWaitEvent(p->compute, p->in_done[k], 0) != cudaSuccess) return ACS_E_CUDA;
    // the state was replaced: restart the step count (acs_set_state's bookkeeping)
    if (int rc = acs_set_state(c, v.phi)) return rc;
    double* d_log = nullptr;
    int64_t entries = 0;
    if (int rc = ctx_enqueue_logged(c, n_steps, every, &d_log, &entries)) return rc;
    if (cudaEventRecord(p->comp_done[k], p->compute) != cudaSuccess) return ACS_E_CUDA;
    if (cudaStreamWaitEvent(p->out, p->comp_done[k], 0) != cudaSuccess) return ACS_E_CUDA;
    if (cudaMemcpyAsync(h_out, v.phi, sb, cudaMemcpyDeviceToHost, p->out) != cudaSuccess) return ACS_E_CUDA;
    if (entries > 0 && cudaMemcpyAsync(h_log, d_log, sizeof(double) * 2 * entries, cudaMemcpyDeviceToHost,
                                       p->out) != cudaSuccess)
        return ACS_E_CUDA;
    if (cudaEventRecord(p->out_done[k], p->out) != cudaSuccess) return ACS_E_CUDA;
    p->pending.push_back(acs_pipe::Pending{h_log, entries});
    p->next = k + 1 == p->slots ? 0 : k + 1;
    return ACS_OK;
}

ACS_API int acs_pipe_wait(acs_pipe* p) {
    if (!p) return ACS_E_INVAL;
    if (!p->bound) return ACS_OK;
    if (cudaStreamSynchronize(p->out) != cudaSuccess || cudaStreamSynchronize(p->compute) != cudaSuccess)
        return ACS_E_CUDA;
    int rc = ACS_OK;
    for (int k = 0; k < p->slots; ++k)
        if (int e = ctx_check_err(p->ctx[k])) rc = rc ? rc : e;
    if (rc) {
        p->pending.clear();
        return rc;
    }
    bool finite = true;
    for (const auto& j : p->pending)
        for (int64_t i = 0; i < 2 * j.entries; ++i) finite = finite && std::isfinite(j.log[i]);
    p->pending.clear();
    return finite ? ACS_OK : ACS_E_NONFINITE;
}

ACS_API void acs_pipe_destroy(acs_pipe* p) {
    if (!p) return;
    if (p->bound) {
        cudaStreamSynchronize(p->out);
        cudaStreamSynchronize(p->in);
    }
    for (int k = 0; k < p->slots; ++k) acs_destroy(p->ctx[k]);
    release_streams(p);
    delete p;
}

}  // extern "C"
