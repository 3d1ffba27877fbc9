// lbm_noalloc.cu -- lbm_build_tiles_noalloc: the tile-map builder without any device
// allocation.
//
// Some callers cannot call cudaMalloc: code that runs inside a framework whose caching
// allocator has reserved the device memory up front, or a real-time / embedded host
// that forbids allocation after its start-up phase. They own their inputs and outputs
// already and only need the builder's temporary storage to come from somewhere else.
// Here that storage lives in one file-scope device array that every GPU loading the
// library holds until the process exits; the entry point reuses the tile_flag -> scan
// -> scatter kernels of lbm_create with pointers into that array.
#include <mutex>

#include "lbm_internal.cuh"

namespace {

constexpr int64_t kMaxTiles = LBM_NOALLOC_MAX_TILES;                  // 2^22 tiles
constexpr size_t kFlagsBytes = (size_t)kMaxTiles;                     // one byte per tile
constexpr size_t kSumsOffset = kFlagsBytes;                           // 256-aligned
constexpr size_t kSumsBytes = (size_t)((kMaxTiles + 1023) / 1024) * sizeof(int64_t);
constexpr size_t kCountOffset = kSumsOffset + kSumsBytes;             // int64 tile count
constexpr size_t kBadOffset = kCountOffset + 256;                      // int error flag
constexpr size_t kScratchBytes = kBadOffset + 256;

static __device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
void* g_scratch_ptr[kMaxDevices] = {};

}  // namespace

extern "C" lbm_status lbm_build_tiles_noalloc(const uint8_t* node_type, int nx, int ny, int nz,
                                              int32_t* tile_map, uint32_t* non_empty, int64_t* n_tiles,
                                              void* stream) {
    if (!node_type || !tile_map || !non_empty || !n_tiles) return LBM_EINVAL;
    if (nx < 1 || ny < 1 || nz < 1) return LBM_EINVAL;
    // widened before the rounding-up add: nx near INT_MAX must not wrap
    const int64_t Tx = ((int64_t)nx + 3) / 4, Ty = ((int64_t)ny + 3) / 4, Tz = ((int64_t)nz + 3) / 4;
    if (Tx > kMaxTiles || Ty > kMaxTiles || Tz > kMaxTiles) return LBM_EUNSUPPORTED;
    const int64_t nT = Tx * Ty * Tz;   // each factor <= 2^22, so no overflow
    if (nT <= 0) return LBM_EINVAL;
    if (nT > kMaxTiles) return LBM_EUNSUPPORTED;   // beyond the static scratch: use lbm_create
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return LBM_ECUDA;
    if (dev < 0 || dev >= kMaxDevices) return LBM_EUNSUPPORTED;
    unsigned char* base = nullptr;
    {
        // Set-up, once per device with that device current: the device address of the
        // static array (its host-side name is only a stand-in for the symbol).
        std::lock_guard<std::mutex> lock(g_mu);
        if (!g_scratch_ptr[dev]) {
            void* p = nullptr;
            e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
            if (e != cudaSuccess) return LBM_ECUDA;
            g_scratch_ptr[dev] = p;
        }
        base = static_cast<unsigned char*>(g_scratch_ptr[dev]);
    }
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    uint8_t* flags = base;
    int64_t* sums = reinterpret_cast<int64_t*>(base + kSumsOffset);
    int64_t* d_count = reinterpret_cast<int64_t*>(base + kCountOffset);
    int* d_bad = reinterpret_cast<int*>(base + kBadOffset);
    // The array keeps the previous call's contents. Flags, block sums and the count are
    // rewritten in full below; only the error flag has to start at zero.
    e = cudaMemsetAsync(d_bad, 0, sizeof(int), st);
    if (e == cudaSuccess) e = lbm::launch_tile_flags(node_type, nx, ny, nz, (int)Tx, (int)Ty, (int)Tz, flags, d_bad, st);
    if (e == cudaSuccess)
        e = lbm::launch_scan_flags(flags, nT, tile_map, non_empty, d_count, sums, lbm::scan_block_count(nT), st);
    int64_t count = 0;
    int bad = 0;
    if (e == cudaSuccess) e = cudaMemcpyAsync(&count, d_count, sizeof(count), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(&bad, d_bad, sizeof(bad), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return LBM_ECUDA;
    if (bad) return LBM_EINVAL;   // node types outside 0..3
    *n_tiles = count;
    return LBM_OK;
}
