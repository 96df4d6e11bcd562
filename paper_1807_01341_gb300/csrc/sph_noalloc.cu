// Allocation-free variant of the cell ordering done by sph_build_cells.
//
// sph_cell_order_noalloc computes the same stable (cell, Morton code) order
// as sph_build_cells, for up to NOALLOC_MAX_PARTICLES particles, without
// allocating: its sort buffers live in one file-scope __device__ array that
// every GPU loading this library holds until the process exits.  Its keys
// kernel reads the positions without writing them back (sph_build_cells also
// wraps them in place); the radix sort is the library's own.
#include <cstddef>
#include <mutex>

#include "sph_internal.cuh"

namespace sph {
namespace {

constexpr int NOALLOC_MAX = 1 << 16;                       // particles per call
constexpr int NOALLOC_TILES = (NOALLOC_MAX + 4095) / 4096;  // radix-sort tiles of 4096 keys
// byte offsets inside the scratch array (each a multiple of 256)
constexpr size_t OFF_KEYS0 = 0;
constexpr size_t OFF_KEYS1 = OFF_KEYS0 + sizeof(unsigned long long) * NOALLOC_MAX;
constexpr size_t OFF_VALS0 = OFF_KEYS1 + sizeof(unsigned long long) * NOALLOC_MAX;
constexpr size_t OFF_VALS1 = OFF_VALS0 + sizeof(unsigned int) * NOALLOC_MAX;
constexpr size_t OFF_HIST = OFF_VALS1 + sizeof(unsigned int) * NOALLOC_MAX;
constexpr size_t OFF_SCAN = OFF_HIST + sizeof(unsigned int) * 256 * NOALLOC_TILES;
constexpr size_t SCRATCH_BYTES = OFF_SCAN + sizeof(unsigned int) * 4096;  // 1.6 MB

static __device__ __align__(256) unsigned char g_noalloc_scratch[SCRATCH_BYTES];

// Device address of the scratch array for each device, looked up once per
// device (with that device current) on its first call and kept for the life
// of the process (a cudaDeviceReset on that device invalidates it; the header
// asks callers not to call again after one).
std::mutex g_mu;
void *g_addr[64] = {};

cudaError_t scratch_address(void **out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lock(g_mu);
  if (!g_addr[dev]) {
    void *p = nullptr;
    e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) return e;
    g_addr[dev] = p;
  }
  *out = g_addr[dev];
  return cudaSuccess;
}

// --- keys: the same FP64 arithmetic as the build's keys, positions unchanged
__device__ __forceinline__ double wrap_box_ro(double x, double box) {
  if (x < 0.0) x = __dadd_rn(x, box);
  if (x >= box) x = __dsub_rn(x, box);
  return x;
}

__device__ __forceinline__ int axis_cell_ro(double x, double w, int nc) {
  int c = (int)floor(__ddiv_rn(x, w));
  return c < 0 ? 0 : (c > nc - 1 ? nc - 1 : c);
}

__device__ __forceinline__ unsigned long long axis_morton_ro(double x, int c, double w) {
  double t = __ddiv_rn(__dsub_rn(x, __dmul_rn((double)c, w)), w);
  t = __dmul_rn(t, (double)(1 << MORTON_BITS));
  double ft = floor(t);
  long long q = (long long)ft;
  if (ft < 0.0) q = 0;
  if (q > (1 << MORTON_BITS) - 1) q = (1 << MORTON_BITS) - 1;
  return (unsigned long long)q;
}

__device__ __forceinline__ unsigned long long spread3_ro(unsigned long long v) {
  unsigned long long r = 0;
#pragma unroll
  for (int b = 0; b < MORTON_BITS; b++) r |= ((v >> b) & 1ull) << (3 * b);
  return r;
}

__global__ void k_cell_keys_ro(const double *__restrict__ xs, const double *__restrict__ ys,
                               const double *__restrict__ zs, int n, double box, int nc, double w,
                               unsigned long long *__restrict__ keys,
                               unsigned int *__restrict__ vals) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const double x = wrap_box_ro(xs[i], box), y = wrap_box_ro(ys[i], box), z = wrap_box_ro(zs[i], box);
  const int cx = axis_cell_ro(x, w, nc), cy = axis_cell_ro(y, w, nc), cz = axis_cell_ro(z, w, nc);
  const unsigned long long cid = ((unsigned long long)cx * nc + cy) * nc + cz;
  const unsigned long long mort = (spread3_ro(axis_morton_ro(x, cx, w)) << 2) |
                                  (spread3_ro(axis_morton_ro(y, cy, w)) << 1) |
                                  spread3_ro(axis_morton_ro(z, cz, w));
  keys[i] = (cid << KEY_MORTON_BITS) | mort;
  vals[i] = (unsigned int)i;
}

}  // namespace
}  // namespace sph

extern "C" int sph_cell_order_noalloc(const double *x, const double *y, const double *z, int64_t n,
                                      double box, int n_cells_per_axis, int32_t *perm,
                                      void *stream) {
  using namespace sph;
  if (n < 0 || n > NOALLOC_MAX || !(box > 0.0) || n_cells_per_axis < 1 || n_cells_per_axis > 255)
    return SPH_ERR_ARG;
  if (n > 0 && (!x || !y || !z || !perm)) return SPH_ERR_ARG;
  void *base = nullptr;
  if (scratch_address(&base) != cudaSuccess) return SPH_ERR_CUDA;
  if (n == 0) return SPH_OK;
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  unsigned char *s = static_cast<unsigned char *>(base);
  auto *keys0 = reinterpret_cast<unsigned long long *>(s + OFF_KEYS0);
  auto *keys1 = reinterpret_cast<unsigned long long *>(s + OFF_KEYS1);
  auto *vals0 = reinterpret_cast<unsigned int *>(s + OFF_VALS0);
  auto *vals1 = reinterpret_cast<unsigned int *>(s + OFF_VALS1);
  auto *hist = reinterpret_cast<unsigned int *>(s + OFF_HIST);
  auto *scan = reinterpret_cast<unsigned int *>(s + OFF_SCAN);
  const int nc = n_cells_per_axis;
  const double w = box / (double)nc;
  const long long n_cells = (long long)nc * nc * nc;
  note_launches(1);
  k_cell_keys_ro<<<(int)((n + 255) / 256), 256, 0, st>>>(x, y, z, (int)n, box, nc, w, keys0, vals0);
  if (cudaGetLastError() != cudaSuccess) return SPH_ERR_CUDA;
  int cell_bits = 1;
  while ((1LL << cell_bits) < n_cells) cell_bits++;
  // every buffer the sort reads is written first in each call: nothing to clear
  bool alt = false;
  if (radix_sort_pairs(keys0, vals0, keys1, vals1, (int)n, KEY_MORTON_BITS + cell_bits, hist, scan,
                       256 * NOALLOC_TILES, &alt, st, nullptr) != cudaSuccess)
    return SPH_ERR_CUDA;
  if (cudaMemcpyAsync(perm, alt ? vals1 : vals0, sizeof(int32_t) * (size_t)n,
                      cudaMemcpyDeviceToDevice, st) != cudaSuccess)
    return SPH_ERR_CUDA;
  return SPH_OK;
}
