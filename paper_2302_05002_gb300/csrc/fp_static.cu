// fp_static.cu -- fp_bounds_decimate_static: the fused bounds + preview pass
// without a caller workspace.
//
// Some callers cannot call cudaMalloc: a host application whose device memory
// is owned and budgeted by another allocator (an engine or a plugin host), or a
// real-time loop that must not wait on an allocator.  For them the scratch the
// pass needs (per-block partial extents, one look-back word per tile, a tile
// counter) lives in a file-scope device array that every GPU loading this
// library holds until the process exits.
#include <mutex>
#include "fp_internal.cuh"

namespace fp {

constexpr size_t kStaticScratchBytes = 1024 * 1024;
constexpr uint64_t kStaticMaxPoints = 1ull << 27;   // 134,217,728 points

static __device__ __align__(256) unsigned char g_static_scratch[kStaticScratchBytes];

static std::mutex g_static_mu;
static void* g_static_ptr[64];

// Device address of the scratch array for the current device, looked up once
// per device with that device current (the host-side name of the array is not
// a device address and must never reach a kernel).
static fp_status static_scratch(void** out)
{
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return FP_ERR_CUDA;
    std::lock_guard<std::mutex> lk(g_static_mu);
    if (!g_static_ptr[dev]) {
        void* p = nullptr;
        if (cudaGetSymbolAddress(&p, g_static_scratch) != cudaSuccess || p == nullptr) return FP_ERR_CUDA;
        g_static_ptr[dev] = p;
    }
    *out = g_static_ptr[dev];
    return FP_OK;
}

}  // namespace fp

using namespace fp;

extern "C" fp_status fp_bounds_decimate_static(const fp_point* d_pts, uint64_t n, fp_cube* d_cube,
                                               uint64_t first_index, uint32_t modulus, fp_point* d_out,
                                               uint64_t out_cap, uint64_t* d_out_count, cudaStream_t stream)
{
    if (!d_cube || !d_out_count || (n && (!d_pts || (out_cap && !d_out))) || modulus < 1) return FP_ERR_INVALID;
    if (n > kStaticMaxPoints) return FP_ERR_TOO_LARGE;
    if ((n && (reinterpret_cast<uintptr_t>(d_pts) & 15u)) || (d_out && (reinterpret_cast<uintptr_t>(d_out) & 15u)))
        return FP_ERR_ALIGN;
    void* scratch = nullptr;
    fp_status s = static_scratch(&scratch);
    if (s != FP_OK) return s;
    Workspace ws;
    s = make_workspace(scratch, kStaticScratchBytes, 0, ws);
    if (s != FP_OK) return s;
    if (bounds_ws_bytes(n, ws.num_sms) > kStaticScratchBytes) return FP_ERR_TOO_LARGE;
    return launch_bounds_decimate(d_pts, n, d_cube, true, true, first_index, modulus, d_out, out_cap, d_out_count,
                                  ws, stream) == cudaSuccess
               ? FP_OK
               : FP_ERR_CUDA;
}
