// Tensor maps (TMA descriptors) of a population array, encoded on the host
// through the driver entry point so that the library needs no link against
// the driver library.
#include <cudaTypedefs.h>

#include <cstring>
#include <mutex>

#include "elbm_internal.h"

namespace elbm {

namespace {

PFN_cuTensorMapEncodeTiled_v12000 encode_fn()
{
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    static std::once_flag once;
    std::call_once(once, [] {
        void* ptr = nullptr;
        cudaDriverEntryPointQueryResult q{};
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &ptr, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(ptr);
        else
            (void)cudaGetLastError();
    });
    return fn;
}

}  // namespace

cudaError_t encode_uncached(const Solver& s, const void* f, int tile_y, CUtensorMap* tile, CUtensorMap* row);

// The maps of array f: from the solver's cache (two arrays deep, keyed by
// address and tile height), else encoded and cached.
cudaError_t encode_population_maps(const Solver& s, const void* f, int tile_y, CUtensorMap* tile, CUtensorMap* row)
{
    static_assert(sizeof(CUtensorMap) == 128, "a tensor map is 128 bytes");
    for (int k = 0; k < 2; ++k)
        if (s.tmap_f[k] == f && s.tmap_tile_y[k] == tile_y) {
            std::memcpy(tile, s.tmap[k][0], sizeof(CUtensorMap));
            std::memcpy(row, s.tmap[k][1], sizeof(CUtensorMap));
            return cudaSuccess;
        }
    const cudaError_t e = encode_uncached(s, f, tile_y, tile, row);
    if (e == cudaSuccess) {
        const int k = s.tmap_next;
        s.tmap_next ^= 1;
        std::memcpy(s.tmap[k][0], tile, sizeof(CUtensorMap));
        std::memcpy(s.tmap[k][1], row, sizeof(CUtensorMap));
        s.tmap_f[k] = f;
        s.tmap_tile_y[k] = tile_y;
    }
    return e;
}

// Layout f[i][z][y][x] as a 4-D tensor (x, y, z, i) of 4- or 2-byte elements;
// boxes of 32 x tile_y x 1 x 27 (the tile of one plane) and 32 x 1 x 1 x 27 (one
// ring row).  Strides are multiples of 16 bytes when nx * element size is.
cudaError_t encode_uncached(const Solver& s, const void* f, int tile_y, CUtensorMap* tile, CUtensorMap* row)
{
    const PFN_cuTensorMapEncodeTiled_v12000 fn = encode_fn();
    if (!fn || s.D != 3) return cudaErrorNotSupported;
    const cuuint64_t es = storage_bytes(s.storage);
    const cuuint64_t dims[4] = {(cuuint64_t)s.nx, (cuuint64_t)s.ny, (cuuint64_t)s.nz, 27};
    const cuuint64_t strides[3] = {s.nx * es, (cuuint64_t)s.nx * s.ny * es, (cuuint64_t)s.N * es};
    const cuuint32_t box_tile[4] = {32, (cuuint32_t)tile_y, 1, 27}, box_row[4] = {32, 1, 1, 27}, unit[4] = {1, 1, 1, 1};
    const CUtensorMapDataType dt = es == 4 ? CU_TENSOR_MAP_DATA_TYPE_UINT32 : CU_TENSOR_MAP_DATA_TYPE_UINT16;
    for (int k = 0; k < 2; ++k) {
        CUresult r = fn(k == 0 ? tile : row, dt, 4, const_cast<void*>(f), dims, strides, k == 0 ? box_tile : box_row,
                        unit, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                        CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
        if (r != CUDA_SUCCESS) return cudaErrorInvalidValue;
    }
    return cudaSuccess;
}

}  // namespace elbm
