// noalloc.cu -- qsim_prob_noalloc: the FP64 Born-probability reduction for
// callers that must not allocate device memory.
//
// Who needs it: code that owns a state vector in device memory but may not
// call cudaMalloc/cudaFree -- for example a plug-in running inside another
// framework that hands out all device memory from its own fixed pool, or a
// latency-critical loop where an allocation (which can synchronise the whole
// device) is not allowed.  Such a caller passes its state and gets p0/p1 back;
// the reduction's scratch (per-block partial sums and the arrival counter of
// the last-block reduction) comes from the fixed array below instead of an
// allocation.
//
// The scratch array is a file-scope __device__ variable: every GPU that loads
// this library holds its own copy (16.25 KiB) until the process exits.  Host
// code cannot use the array's name as a device address, so the first call on
// each device looks the address up with cudaGetSymbolAddress (with that device
// current) and caches it; make that first call on a device before any stream
// capture begins.  All calls on a device share the array and it keeps the
// last call's contents: each call clears the counter and control fields it
// relies on before launching, and calls whose work may overlap on the GPU
// (different streams, or different host threads) race on the array -- the
// caller must order them.
#include <cuda_runtime.h>

#include <cstring>
#include <mutex>

#include "../../include/qsim.h"
#include "kernels.h"

namespace {

// Largest block count of the probability reduction (prob_blocks caps at 1024),
// so every state of 1..34 qubits fits: 1024 (p0, p1) partial pairs + control.
constexpr int kMaxBlocks = 1024;
constexpr size_t kPartialBytes = (size_t)kMaxBlocks * 2 * sizeof(double);
constexpr size_t kScratchBytes = kPartialBytes + 256;
static_assert(sizeof(qsim::MeasCtl) <= 256, "control block must fit the reserved tail");

static __device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
void *g_addr[kMaxDevices] = {nullptr};

}  // namespace

extern "C" QSIM_API qsim_status qsim_prob_noalloc(const void *d_state, int n_qubits, qsim_dtype dtype,
                                                  int qubit, void *stream, double *p0, double *p1) {
    if (!d_state || !p0 || !p1) return QSIM_E_INVAL;
    if (n_qubits < 1 || n_qubits > 34) return QSIM_E_INVAL;  // beyond the static scratch's range
    if (dtype != QSIM_C64 && dtype != QSIM_C128) return QSIM_E_INVAL;
    if (qubit < 0 || qubit >= n_qubits) return QSIM_E_INVAL;
    if (qsim::prob_blocks(n_qubits) > kMaxBlocks) return QSIM_E_INVAL;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) {
        cudaGetLastError();
        return QSIM_E_CUDA;
    }
    // The scratch address below is the current device's copy of the array, so
    // the state and the stream must belong to that device too.
    cudaPointerAttributes pa;
    if (cudaPointerGetAttributes(&pa, d_state) != cudaSuccess) {
        cudaGetLastError();
        return QSIM_E_INVAL;
    }
    if ((pa.type != cudaMemoryTypeDevice && pa.type != cudaMemoryTypeManaged) ||
        (pa.type == cudaMemoryTypeDevice && pa.device != dev))
        return QSIM_E_INVAL;
    if (stream) {
        int sdev = -1;
        if (cudaStreamGetDevice((cudaStream_t)stream, &sdev) != cudaSuccess) {
            cudaGetLastError();
            return QSIM_E_INVAL;
        }
        if (sdev != dev) return QSIM_E_INVAL;
    }
    void *base = nullptr;
    {
        std::lock_guard<std::mutex> lk(g_mu);
        if (!g_addr[dev]) {
            void *ptr = nullptr;
            cudaError_t e = cudaGetSymbolAddress(&ptr, g_noalloc_scratch);
            if (e != cudaSuccess || !ptr) {
                cudaGetLastError();
                return QSIM_E_CUDA;
            }
            g_addr[dev] = ptr;
        }
        base = g_addr[dev];
    }
    double *partials = reinterpret_cast<double *>(base);
    qsim::MeasCtl *ctl = reinterpret_cast<qsim::MeasCtl *>(static_cast<unsigned char *>(base) + kPartialBytes);
    cudaStream_t s = (cudaStream_t)stream;
    // status and arrival counter must start at zero for this call
    if (cudaMemsetAsync(ctl, 0, sizeof(qsim::MeasCtl), s) != cudaSuccess) {
        cudaGetLastError();
        return QSIM_E_CUDA;
    }
    if (qsim::launch_prob_only((int)dtype, d_state, n_qubits, qubit, partials, ctl, s) != cudaSuccess) {
        cudaGetLastError();
        return QSIM_E_CUDA;
    }
    double out[2];
    if (cudaMemcpyAsync(out, &ctl->p0, 2 * sizeof(double), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess) {
        cudaGetLastError();
        return QSIM_E_CUDA;
    }
    *p0 = out[0];
    *p1 = out[1];
    return QSIM_OK;
}
