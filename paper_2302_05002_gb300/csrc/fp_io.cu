// fp_io.cu -- the built octree on disk and back, and the cloud digest that
// keys a cache of built clouds.
//
// The converter stitches the local octrees into one global octree that is
// written to a file, and the renderer later loads node points from it on demand
// (Sec. 4.4, Sec. 4.5, Fig. "octree"); a cloud whose octree was built before is
// not built again (Sec. 3, Fig. "pipeline").  One file holds a fixed header,
// the node table (fp_node records in preorder) and the points in the final
// layout (each node's kept points contiguous at node.first), optionally
// followed by the original index of every point.  Device data move through a
// caller-given pinned staging buffer in two halves, so the copy of one piece
// overlaps the file write (or read) of the other.
#include <cstdio>
#include <cstring>
#include <sys/types.h>
#include "fp_internal.cuh"

namespace fp {

namespace {

static_assert(sizeof(fp_file_header) == 160 && sizeof(fp_node) == 40 && sizeof(fp_point) == 16, "file layout");

constexpr char kMagic[8] = {'F', 'P', 'O', 'C', 'T', 'R', 'E', 'E'};
constexpr uint32_t kVersion = 1;
constexpr uint64_t kDigestSalt = 0x5851F42D4C957F2Dull;

uint64_t align_up(uint64_t v, uint64_t a) { return (v + a - 1) / a * a; }

// digest word of point i: mixes the index and both 64-bit halves of the record
__global__ void __launch_bounds__(256) k_digest(const int4* __restrict__ pts, uint64_t n, unsigned long long* out)
{
    uint64_t acc = 0;
    for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (uint64_t)gridDim.x * blockDim.x) {
        const int4 q = __ldg(pts + i);
        const uint64_t a = (uint64_t)(uint32_t)q.x | ((uint64_t)(uint32_t)q.y << 32);
        const uint64_t b = (uint64_t)(uint32_t)q.z | ((uint64_t)(uint32_t)q.w << 32);
        acc += splitmix64(splitmix64(i) ^ splitmix64(a) ^ splitmix64(b ^ kDigestSalt));
    }
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xFFFFFFFFu, acc, o);
    if ((threadIdx.x & 31) == 0 && acc) atomicAdd(out, (unsigned long long)acc);
}

__global__ void k_digest_final(unsigned long long* out, uint64_t n) { *out += n; }

struct File {
    FILE* f = nullptr;
    ~File() { if (f) fclose(f); }
};

bool seek(FILE* f, uint64_t off) { return fseeko(f, (off_t)off, SEEK_SET) == 0; }

// device -> file through the two staging halves
fp_status dev_to_file(FILE* f, const void* d_src, uint64_t bytes, char* stage, size_t half, cudaEvent_t ev[2],
                      cudaStream_t st)
{
    const char* src = static_cast<const char*>(d_src);
    uint64_t done = 0, k = 0;
    uint64_t pending[2] = {0, 0};
    while (done < bytes || pending[0] || pending[1]) {
        const int b = (int)(k & 1);
        if (pending[b]) {   // the piece in this half is on its way: write it out
            if (cudaEventSynchronize(ev[b]) != cudaSuccess) return FP_ERR_CUDA;
            if (fwrite(stage + b * half, 1, pending[b], f) != pending[b]) return FP_ERR_IO;
            pending[b] = 0;
        }
        if (done < bytes) {
            const uint64_t m = std::min<uint64_t>(half, bytes - done);
            if (cudaMemcpyAsync(stage + b * half, src + done, m, cudaMemcpyDeviceToHost, st) != cudaSuccess)
                return FP_ERR_CUDA;
            if (cudaEventRecord(ev[b], st) != cudaSuccess) return FP_ERR_CUDA;
            pending[b] = m;
            done += m;
        }
        ++k;
    }
    return FP_OK;
}

// file -> device through the two staging halves
fp_status file_to_dev(FILE* f, void* d_dst, uint64_t bytes, char* stage, size_t half, cudaEvent_t ev[2],
                      cudaStream_t st)
{
    char* dst = static_cast<char*>(d_dst);
    bool busy[2] = {false, false};
    uint64_t done = 0;
    for (uint64_t k = 0; done < bytes; ++k) {
        const int b = (int)(k & 1);
        if (busy[b] && cudaEventSynchronize(ev[b]) != cudaSuccess) return FP_ERR_CUDA;   // half free again
        const uint64_t m = std::min<uint64_t>(half, bytes - done);
        if (fread(stage + b * half, 1, m, f) != m) return FP_ERR_IO;
        if (cudaMemcpyAsync(dst + done, stage + b * half, m, cudaMemcpyHostToDevice, st) != cudaSuccess)
            return FP_ERR_CUDA;
        if (cudaEventRecord(ev[b], st) != cudaSuccess) return FP_ERR_CUDA;
        busy[b] = true;
        done += m;
    }
    for (int b = 0; b < 2; ++b)
        if (busy[b] && cudaEventSynchronize(ev[b]) != cudaSuccess) return FP_ERR_CUDA;
    return FP_OK;
}

struct Events {
    cudaEvent_t e[2] = {nullptr, nullptr};
    bool ok = false;
    Events()
    {
        ok = cudaEventCreateWithFlags(&e[0], cudaEventDisableTiming) == cudaSuccess &&
             cudaEventCreateWithFlags(&e[1], cudaEventDisableTiming) == cudaSuccess;
    }
    ~Events()
    {
        for (cudaEvent_t x : e)
            if (x) cudaEventDestroy(x);
    }
};

fp_status read_header(FILE* f, fp_file_header* h)
{
    if (!seek(f, 0) || fread(h, sizeof(*h), 1, f) != 1) return FP_ERR_IO;
    if (memcmp(h->magic, kMagic, 8) != 0 || h->version != kVersion || h->header_bytes != sizeof(fp_file_header))
        return FP_ERR_INVALID;
    return FP_OK;
}

}  // namespace

}  // namespace fp

using namespace fp;

extern "C" {

fp_status fp_cloud_digest(const fp_point* d_pts, uint64_t n, uint64_t* d_digest, cudaStream_t stream)
{
    if (!d_digest || (n && !d_pts)) return FP_ERR_INVALID;
    if (n && (reinterpret_cast<uintptr_t>(d_pts) & 15u)) return FP_ERR_ALIGN;
    int dev = 0, sms = 152;
    if (cudaGetDevice(&dev) != cudaSuccess) return FP_ERR_CUDA;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (cudaMemsetAsync(d_digest, 0, sizeof(uint64_t), stream) != cudaSuccess) return FP_ERR_CUDA;
    if (n) {
        const int grid = (int)std::min<uint64_t>((n + 255) / 256, (uint64_t)sms * 8);
        k_digest<<<grid, 256, 0, stream>>>(reinterpret_cast<const int4*>(d_pts), n,
                                           reinterpret_cast<unsigned long long*>(d_digest));
    }
    k_digest_final<<<1, 1, 0, stream>>>(reinterpret_cast<unsigned long long*>(d_digest), n);
    return cudaGetLastError() == cudaSuccess ? FP_OK : FP_ERR_CUDA;
}

static fp_status octree_save(const char* path, const fp_params* h_prm, const fp_cube* d_cube, const fp_node* d_nodes,
                         const uint32_t* d_num_nodes, const fp_point* d_final, const uint32_t* d_final_perm,
                         uint64_t n, uint64_t digest, void* h_staging, size_t staging_bytes, cudaStream_t stream)
{
    if (!path || !h_prm || !d_cube || !d_num_nodes || !h_staging || (n && !d_final)) return FP_ERR_INVALID;
    const size_t half = staging_bytes / 2 / 16 * 16;
    if (half < 4096) return FP_ERR_WORKSPACE;
    fp_file_header h;
    memset(&h, 0, sizeof(h));
    memcpy(h.magic, kMagic, 8);
    h.version = kVersion;
    h.header_bytes = sizeof(fp_file_header);
    h.prm = *h_prm;
    h.n = n;
    h.digest = digest;
    uint32_t M = 0;
    if (cudaMemcpyAsync(&M, d_num_nodes, sizeof(M), cudaMemcpyDeviceToHost, stream) != cudaSuccess) return FP_ERR_CUDA;
    if (cudaMemcpyAsync(&h.cube, d_cube, sizeof(fp_cube), cudaMemcpyDeviceToHost, stream) != cudaSuccess)
        return FP_ERR_CUDA;
    if (cudaStreamSynchronize(stream) != cudaSuccess) return FP_ERR_CUDA;
    if (M && !d_nodes) return FP_ERR_INVALID;
    h.num_nodes = M;
    h.flags = d_final_perm ? FP_FILE_HAS_PERM : 0u;
    h.nodes_offset = align_up(sizeof(fp_file_header), 4096);
    h.points_offset = align_up(h.nodes_offset + (uint64_t)M * sizeof(fp_node), 4096);
    h.perm_offset = d_final_perm ? h.points_offset + n * sizeof(fp_point) : 0;
    File F;
    F.f = fopen(path, "wb");
    if (!F.f) return FP_ERR_IO;
    Events E;
    if (!E.ok) return FP_ERR_CUDA;
    char* stage = static_cast<char*>(h_staging);
    fp_status s;
    if (fwrite(&h, sizeof(h), 1, F.f) != 1) return FP_ERR_IO;
    if (!seek(F.f, h.nodes_offset)) return FP_ERR_IO;
    if ((s = dev_to_file(F.f, d_nodes, (uint64_t)M * sizeof(fp_node), stage, half, E.e, stream))) return s;
    if (!seek(F.f, h.points_offset)) return FP_ERR_IO;
    if ((s = dev_to_file(F.f, d_final, n * sizeof(fp_point), stage, half, E.e, stream))) return s;
    if (d_final_perm && (s = dev_to_file(F.f, d_final_perm, n * sizeof(uint32_t), stage, half, E.e, stream)))
        return s;
    if (fflush(F.f) != 0) return FP_ERR_IO;
    const int rc = fclose(F.f);
    F.f = nullptr;
    return rc == 0 ? FP_OK : FP_ERR_IO;
}

fp_status fp_octree_read_header(const char* path, fp_file_header* h_hdr)
{
    if (!path || !h_hdr) return FP_ERR_INVALID;
    File F;
    F.f = fopen(path, "rb");
    if (!F.f) return FP_ERR_IO;
    return read_header(F.f, h_hdr);
}

static fp_status octree_load(const char* path, fp_node* d_nodes, uint32_t node_cap, fp_point* d_points,
                         uint32_t* d_perm, uint64_t first, uint64_t count, void* h_staging, size_t staging_bytes,
                         cudaStream_t stream)
{
    if (!path || !h_staging) return FP_ERR_INVALID;
    const size_t half = staging_bytes / 2 / 16 * 16;
    if (half < 4096) return FP_ERR_WORKSPACE;
    File F;
    F.f = fopen(path, "rb");
    if (!F.f) return FP_ERR_IO;
    fp_file_header h;
    fp_status s = read_header(F.f, &h);
    if (s) return s;
    if (first > h.n || count > h.n - first) return FP_ERR_INVALID;
    if (d_perm && !(h.flags & FP_FILE_HAS_PERM)) return FP_ERR_INVALID;
    if (d_nodes && h.num_nodes > node_cap) return FP_ERR_CAPACITY;
    Events E;
    if (!E.ok) return FP_ERR_CUDA;
    char* stage = static_cast<char*>(h_staging);
    if (d_nodes) {
        if (!seek(F.f, h.nodes_offset)) return FP_ERR_IO;
        if ((s = file_to_dev(F.f, d_nodes, (uint64_t)h.num_nodes * sizeof(fp_node), stage, half, E.e, stream)))
            return s;
    }
    if (d_points && count) {
        if (!seek(F.f, h.points_offset + first * sizeof(fp_point))) return FP_ERR_IO;
        if ((s = file_to_dev(F.f, d_points, count * sizeof(fp_point), stage, half, E.e, stream))) return s;
    }
    if (d_perm && count) {
        if (!seek(F.f, h.perm_offset + first * sizeof(uint32_t))) return FP_ERR_IO;
        if ((s = file_to_dev(F.f, d_perm, count * sizeof(uint32_t), stage, half, E.e, stream))) return s;
    }
    return FP_OK;
}

fp_status fp_octree_save(const char* path, const fp_params* h_prm, const fp_cube* d_cube, const fp_node* d_nodes,
                         const uint32_t* d_num_nodes, const fp_point* d_final, const uint32_t* d_final_perm,
                         uint64_t n, uint64_t digest, void* h_staging, size_t staging_bytes, cudaStream_t stream)
{
    fp_status s = octree_save(path, h_prm, d_cube, d_nodes, d_num_nodes, d_final, d_final_perm, n, digest, h_staging,
                              staging_bytes, stream);
    if (s != FP_OK) cudaStreamSynchronize(stream);   // no copy into the staging buffer outlives the call
    return s;
}

fp_status fp_octree_load(const char* path, fp_node* d_nodes, uint32_t node_cap, fp_point* d_points,
                         uint32_t* d_perm, uint64_t first, uint64_t count, void* h_staging, size_t staging_bytes,
                         cudaStream_t stream)
{
    fp_status s = octree_load(path, d_nodes, node_cap, d_points, d_perm, first, count, h_staging, staging_bytes,
                              stream);
    if (s != FP_OK) cudaStreamSynchronize(stream);
    return s;
}

}  // extern "C"
