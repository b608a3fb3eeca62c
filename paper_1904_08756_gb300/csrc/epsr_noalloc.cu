// epsr_noalloc.cu -- the pair histogram of one box without any device allocation.
//
// Some callers cannot allocate device memory at the point where they need a histogram:
// plug-ins that are handed no device memory by a host framework whose caching allocator
// owns the device, or real-time loops that must not call cudaMalloc/cudaFree (which can
// synchronise the whole device) after start-up. For them, epsr_partial_gr_noalloc computes
// the same counts as epsr_partial_gr on a one-box handle, with every piece of working
// memory carved from one file-scope __device__ array of fixed size. The array exists on
// every GPU that loads the library until the process exits.
//
// Host code cannot use the array's name as a device address; its address is obtained
// per device with cudaGetSymbolAddress on the first call made while that device is
// current, and cached for the life of the device's primary context.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <mutex>
#include <vector>

#include "epsr.h"
#include "epsr_device.cuh"
#include "epsr_internal.h"

using namespace epsr;

namespace {

constexpr long long kMaxAtoms = EPSR_NOALLOC_MAX_ATOMS;
constexpr int kMaxCells = 32 * 32 * 32;
constexpr long long kMaxTiles = ((kMaxAtoms + kGrTile - 1) / kGrTile) *
                                ((kMaxAtoms + kGrTile - 1) / kGrTile + 1) / 2;

constexpr size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

// Layout of the scratch array (every region 256-byte aligned).
constexpr size_t kOffBox = 0;
constexpr size_t kOffT = kOffBox + align256(sizeof(BoxDev));
constexpr size_t kOffTiles = kOffT + align256((EPSR_MAX_BINS + 1) * sizeof(long long));
constexpr size_t kOffAtomBox = kOffTiles + align256(kMaxTiles * sizeof(GrTile));
constexpr size_t kOffCoords = kOffAtomBox + align256(kMaxAtoms * sizeof(int));
constexpr size_t kOffScaled = kOffCoords + align256(kMaxAtoms * sizeof(int4));
constexpr size_t kOffSScaled = kOffScaled + align256(kMaxAtoms * sizeof(uint4));
constexpr size_t kOffSCoords = kOffSScaled + align256(kMaxAtoms * sizeof(uint4));
constexpr size_t kOffCount = kOffSCoords + align256(kMaxAtoms * sizeof(int4));
constexpr size_t kOffOffset = kOffCount + align256(kMaxCells * sizeof(int));
constexpr size_t kOffBlock = kOffOffset + align256(kMaxCells * sizeof(int));
constexpr size_t kOffKey = kOffBlock + align256((kMaxCells / 1024 + 1) * sizeof(int));
constexpr size_t kOffRank = kOffKey + align256(kMaxAtoms * sizeof(int));
constexpr size_t kOffIndex = kOffRank + align256(kMaxAtoms * sizeof(int));
constexpr size_t kScratchBytes = kOffIndex + align256(kMaxAtoms * sizeof(int));

__device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];

std::mutex g_mu;
void *g_scratch_addr[256];   // per device ordinal, filled on first use

int scratch_address(unsigned char **out)
{
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return set_cuda_error(e, "cudaGetDevice");
    if (dev < 0 || dev >= 256) return set_error(EPSR_EINVAL, "device ordinal %d not supported", dev);
    std::lock_guard<std::mutex> lock(g_mu);
    if (!g_scratch_addr[dev]) {
        void *p = nullptr;
        e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess) return set_cuda_error(e, "cudaGetSymbolAddress(scratch)");
        g_scratch_addr[dev] = p;
    }
    *out = static_cast<unsigned char *>(g_scratch_addr[dev]);
    return EPSR_OK;
}

__global__ void pack_kernel(const int *xyz, const int *type, int4 *coords, int *atom_box, long long n)
{
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x) {
        coords[i] = make_int4(xyz[3 * i], xyz[3 * i + 1], xyz[3 * i + 2], type[i]);
        atom_box[i] = 0;
    }
}

}  // namespace

extern "C" size_t epsr_noalloc_scratch_bytes(void) { return kScratchBytes; }

extern "C" int epsr_partial_gr_noalloc(const int32_t *xyz, const int32_t *type, int64_t n_atoms,
                                       int64_t L_fx, int32_t scale_log2, int32_t n_types,
                                       int32_t bin_p, int32_t bin_q, int32_t n_bins, uint64_t *hist,
                                       epsr_stream_t stream)
{
    if (!xyz || !type || !hist) return set_error(EPSR_EINVAL, "noalloc gr: NULL argument");
    if (n_atoms < 1 || n_atoms > kMaxAtoms)
        return set_error(EPSR_EINVAL, "noalloc gr: n_atoms %lld outside [1, %lld] (the fixed scratch limit)",
                         (long long)n_atoms, kMaxAtoms);
    if (L_fx < 2 || L_fx >= (1LL << 31) || scale_log2 < 10 || scale_log2 > 24 || n_types < 1 ||
        n_types > EPSR_MAX_TYPES || bin_p < 1 || bin_q < 1 || n_bins < 1 || n_bins > EPSR_MAX_BINS)
        return set_error(EPSR_EINVAL, "noalloc gr: box or bin parameters out of range");
    const double S = std::ldexp(1.0, scale_log2);
    const double rmax_fx = (double)n_bins * bin_p / bin_q * S;
    if (rmax_fx * rmax_fx > 4.0e18) return set_error(EPSR_EINVAL, "noalloc gr: bin range too large");
    const int n_pairs = n_types * (n_types + 1) / 2;
    if ((size_t)kGrTile * 32 + (size_t)(n_bins + 1) * 8 + (size_t)n_pairs * n_bins * 4 > 200 * 1024)
        return set_error(EPSR_EINVAL, "noalloc gr: n_pairs * n_bins too large for shared memory");
    for (long long i = 0; i < n_atoms; ++i) {
        if (type[i] < 0 || type[i] >= n_types)
            return set_error(EPSR_EINVAL, "noalloc gr: type[%lld] = %d out of range", i, type[i]);
        for (int c = 0; c < 3; ++c)
            if (xyz[3 * i + c] < 0 || xyz[3 * i + c] >= L_fx)
                return set_error(EPSR_EINVAL, "noalloc gr: coordinate %lld outside [0, L_fx)", 3 * i + c);
    }
    unsigned char *base = nullptr;
    int rc = scratch_address(&base);
    if (rc) return rc;
    cudaStream_t s = (cudaStream_t)stream;

    // host-side tables (exact thresholds T[k] = ceil((k p S / q)^2), tile work list)
    BoxDev bx;
    memset(&bx, 0, sizeof(bx));
    bx.n_atoms = (int)n_atoms;
    bx.L = (int)L_fx;
    bx.n_types = n_types;
    bx.n_pairs = n_pairs;
    bx.n_bins = n_bins;
    bx.inv_dr_fx = (float)((double)bin_q / ((double)bin_p * S));
    std::vector<long long> T(n_bins + 1);
    const unsigned __int128 q2 = (unsigned __int128)bin_q * bin_q;
    for (int k = 0; k <= n_bins; ++k) {
        const unsigned __int128 num = ((unsigned __int128)k * k * bin_p * bin_p) << (2 * scale_log2);
        T[k] = (long long)((num + q2 - 1) / q2);
    }
    bx.tmax = T[n_bins];
    bx.tmax_lo = (float)((double)bx.tmax * (1.0 - 0x1p-20));
    bx.tmax_hi = (float)((double)bx.tmax * (1.0 + 0x1p-20));
    set_prefilter(bx);
    int nc = (int)std::floor((double)L_fx / S / 3.0);
    nc = std::max(1, std::min(nc, 32));
    int p2 = 1;
    while (p2 < nc) p2 <<= 1;
    bx.cells = nc;
    bx.cells_p3 = p2 * p2 * p2;
    std::vector<GrTile> tiles;
    const int nt = (int)((n_atoms + kGrTile - 1) / kGrTile);
    for (int i = 0; i < nt; ++i)
        for (int j = i; j < nt; ++j) tiles.push_back(GrTile{0, i, j, 0});

    BoxDev *d_box = reinterpret_cast<BoxDev *>(base + kOffBox);
    long long *d_T = reinterpret_cast<long long *>(base + kOffT);
    GrTile *d_tiles = reinterpret_cast<GrTile *>(base + kOffTiles);
    int *d_atom_box = reinterpret_cast<int *>(base + kOffAtomBox);
    int4 *d_coords = reinterpret_cast<int4 *>(base + kOffCoords);
    uint4 *d_scaled = reinterpret_cast<uint4 *>(base + kOffScaled);
    uint4 *d_sscaled = reinterpret_cast<uint4 *>(base + kOffSScaled);
    int4 *d_scoords = reinterpret_cast<int4 *>(base + kOffSCoords);
    SortScratch sc;
    sc.count = reinterpret_cast<int *>(base + kOffCount);
    sc.offset = reinterpret_cast<int *>(base + kOffOffset);
    sc.block = reinterpret_cast<int *>(base + kOffBlock);
    sc.key = reinterpret_cast<int *>(base + kOffKey);
    sc.rank = reinterpret_cast<int *>(base + kOffRank);
    sc.index = reinterpret_cast<int *>(base + kOffIndex);

    // Inputs go into the tail of the coordinate regions before packing: xyz (12 B/atom)
    // into the sorted-coordinate region, types into the rank region.
    int *d_xyz_in = reinterpret_cast<int *>(d_scoords);
    int *d_type_in = sc.rank;
    cudaError_t e;
    if ((e = cudaMemcpyAsync(d_box, &bx, sizeof(bx), cudaMemcpyHostToDevice, s)) != cudaSuccess ||
        (e = cudaMemcpyAsync(d_T, T.data(), T.size() * sizeof(long long), cudaMemcpyHostToDevice, s)) != cudaSuccess ||
        (e = cudaMemcpyAsync(d_tiles, tiles.data(), tiles.size() * sizeof(GrTile), cudaMemcpyHostToDevice, s)) != cudaSuccess ||
        (e = cudaMemcpyAsync(d_xyz_in, xyz, (size_t)n_atoms * 3 * sizeof(int), cudaMemcpyHostToDevice, s)) != cudaSuccess ||
        (e = cudaMemcpyAsync(d_type_in, type, (size_t)n_atoms * sizeof(int), cudaMemcpyHostToDevice, s)) != cudaSuccess)
        return set_cuda_error(e, "noalloc gr: upload");
    const int grid = (int)std::min<long long>((n_atoms + 255) / 256, 4096);
    pack_kernel<<<grid, 256, 0, s>>>(d_xyz_in, d_type_in, d_coords, d_atom_box, n_atoms);
    note_launch();
    if ((e = cudaGetLastError()) != cudaSuccess) return set_cuda_error(e, "noalloc gr: pack");
    if ((rc = launch_scale_coords(d_box, d_atom_box, d_coords, d_scaled, n_atoms, s))) return rc;
    if ((rc = launch_spatial_sort(d_box, d_atom_box, d_scaled, d_coords, n_atoms, bx.cells_p3, 0, sc,
                                  d_sscaled, d_scoords, nullptr, s)))
        return rc;
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    GrArgs a;
    a.boxes = d_box;
    a.coords = d_scoords;
    a.scaled = d_sscaled;
    a.thresholds = d_T;
    a.tiles = d_tiles;
    a.tile_begin = 0;
    a.tile_end = (long long)tiles.size();
    a.hist = (unsigned long long *)hist;
    a.max_pairs_bins = n_pairs * n_bins;
    a.max_bins1 = n_bins + 1;
    return launch_partial_gr(a, (int)std::max<long long>(1, std::min<long long>(a.tile_end, 4LL * sms)), s);
}
