// hacc_bin_noalloc: the binning call for callers that cannot allocate device
// memory.  Its scratch space lives in one fixed array in the library's own
// device memory instead of a caller-supplied workspace.
#include <mutex>

#include "hacc_common.cuh"

namespace {

// HACC_BIN_NOALLOC_BYTES (9 MiB): hacc_bin's scratch, about 30 bytes per
// particle whatever the number of cells (262,144 particles fit).
constexpr size_t NOALLOC_BIN_BYTES = HACC_BIN_NOALLOC_BYTES;

// Loaded with the library onto every device that runs it, and held until the
// process exits.  Every call shares it.
static __device__ __align__(256) unsigned char g_bin_scratch[NOALLOC_BIN_BYTES];

constexpr int MAX_DEVICES = 64;
std::mutex g_mu;
void *g_scratch_addr[MAX_DEVICES] = {};

// Device address of g_bin_scratch on the current device.  In host code the
// symbol's name is only a host-side stand-in, so the address is looked up
// once per device (with that device current) and remembered.  The lookup is
// refused while `st` is being captured into a graph: it would break the
// capture.
int scratch_address(cudaStream_t st, void **out)
{
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= MAX_DEVICES) return HACC_ERR_CUDA;
    std::lock_guard<std::mutex> lock(g_mu);
    if (!g_scratch_addr[dev]) {
        cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
        if (cudaStreamIsCapturing(st, &cap) != cudaSuccess) {
            (void)cudaGetLastError();
            return HACC_ERR_CUDA;
        }
        if (cap != cudaStreamCaptureStatusNone) return HACC_ERR_INVALID;
        void *p = nullptr;
        if (cudaGetSymbolAddress(&p, g_bin_scratch) != cudaSuccess || !p) {
            (void)cudaGetLastError();
            return HACC_ERR_CUDA;
        }
        g_scratch_addr[dev] = p;
    }
    *out = g_scratch_addr[dev];
    return HACC_OK;
}

}  // namespace

extern "C" int hacc_bin_noalloc(const hacc_mesh *mesh, const float *x, const float *y, const float *z,
                                const float *m, const hacc_binned *out, uint32_t *status, void *stream)
{
    if (!mesh) return HACC_ERR_INVALID;
    if (hacc_bin_workspace_size(mesh) > NOALLOC_BIN_BYTES) return HACC_ERR_CAPACITY;
    void *ws = nullptr;
    int rc = scratch_address(hacc::as_stream(stream), &ws);
    if (rc) return rc;
    // hacc_bin writes every scratch word before reading it, so the previous
    // call's contents never leak into this one.
    return hacc_bin(mesh, x, y, z, nullptr, nullptr, nullptr, m, out, ws, NOALLOC_BIN_BYTES, status, stream);
}
