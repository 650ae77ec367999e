// pic_sort_static.cu -- stable sort of one particle set by cell that
// allocates nothing: its (cell, chunk) histogram lives in a fixed device array
// of this library (see pic_sort_by_cell_static in include/pic.h).
//
// Same algorithm as the handle's periodic sort (histogram, one-block scan,
// per-warp stable scatter with __match_any_sync), with plain pointers and the
// scratch taken from g_static_hist instead of a handle.
#include <cuda_runtime.h>

#include <climits>
#include <mutex>

#include "../../include/pic.h"
#include "pic_internal.cuh"

constexpr int kStaticHistInts = 1 << 20;     // 4 MiB of scratch on every device

// The scratch.  Every GPU that loads the library holds it until exit.  Host
// code must not pass this symbol to a kernel: on the host it is only a
// stand-in; its device address comes from cudaGetSymbolAddress below.
static __device__ __align__(256) int g_static_hist[kStaticHistInts];

namespace pic {
namespace {

constexpr int kChunk = 8192;                 // particles per histogram column
constexpr int kThreads = 256;
constexpr int kWarps = kThreads / 32;

struct View {
  const float* z; const float* vx; const float* vy; const float* vz; const uint32_t* id;
  float* zo; float* vxo; float* vyo; float* vzo; uint32_t* ido;
  int* hist;                 // device address of g_static_hist
  long long n;
  int nch;                   // columns: ceil(n / kChunk)
  int Nz;
  float inv_dz;
};

__global__ void __launch_bounds__(kThreads) k_static_hist(View v) {
  extern __shared__ int hs[];
  const int c = blockIdx.x;
  for (int j = threadIdx.x; j < v.Nz; j += blockDim.x) hs[j] = 0;
  __syncthreads();
  const long long i0 = (long long)c * kChunk;
  const long long i1 = min(v.n, i0 + kChunk);
  for (long long i = i0 + threadIdx.x; i < i1; i += blockDim.x) {
    int j;
    float f;
    cell_of(v.z[i], v.inv_dz, v.Nz, j, f);
    atomicAdd(&hs[j], 1);
  }
  __syncthreads();
  // every (cell, column) entry is written, so nothing left by an earlier
  // call is read
  for (int j = threadIdx.x; j < v.Nz; j += blockDim.x) v.hist[(long long)j * v.nch + c] = hs[j];
}

__global__ void __launch_bounds__(1024) k_static_scan(View v) {
  __shared__ int ws[32];
  const long long n = (long long)v.Nz * v.nch;
  int carry = 0;
  for (long long base = 0; base < n; base += blockDim.x) {
    const long long k = base + threadIdx.x;
    const int x = k < n ? v.hist[k] : 0;
    int tot;
    const int ex = block_exclusive_scan<int>(x, &tot, ws);
    if (k < n) v.hist[k] = carry + ex;
    carry += tot;
  }
}

__global__ void __launch_bounds__(kThreads) k_static_scatter(View v) {
  extern __shared__ int woff[];              // [kWarps][Nz]
  const int c = blockIdx.x;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const long long i0 = (long long)c * kChunk;
  const long long i1 = min(v.n, i0 + kChunk);
  const long long w0 = i0 + (long long)warp * (kChunk / kWarps);
  const long long w1 = min(i1, w0 + kChunk / kWarps);
  for (int k = threadIdx.x; k < kWarps * v.Nz; k += blockDim.x) woff[k] = 0;
  __syncthreads();
  int* my = woff + warp * v.Nz;
  for (long long i = w0 + lane; i < w1; i += 32) {
    int j;
    float f;
    cell_of(v.z[i], v.inv_dz, v.Nz, j, f);
    atomicAdd(&my[j], 1);
  }
  __syncthreads();
  for (int j = threadIdx.x; j < v.Nz; j += blockDim.x) {
    int run = v.hist[(long long)j * v.nch + c];
    for (int w = 0; w < kWarps; ++w) {
      const int cnt = woff[w * v.Nz + j];
      woff[w * v.Nz + j] = run;
      run += cnt;
    }
  }
  __syncthreads();
  const unsigned lt = (1u << lane) - 1u;
  for (long long base = w0; base < w1; base += 32) {
    const long long i = base + lane;
    const bool act = i < w1;
    const unsigned am = __ballot_sync(0xffffffffu, act);
    int j = -1;
    if (act) {
      float f;
      cell_of(v.z[i], v.inv_dz, v.Nz, j, f);
    }
    const unsigned peers = __match_any_sync(0xffffffffu, j) & am;
    int pos = 0;
    if (act) pos = my[j] + __popc(peers & lt);
    __syncwarp();
    if (act && (peers & lt) == 0u) my[j] += __popc(peers);
    __syncwarp();
    if (act) {
      v.zo[pos] = v.z[i];
      v.vxo[pos] = v.vx[i];
      v.vyo[pos] = v.vy[i];
      v.vzo[pos] = v.vz[i];
      v.ido[pos] = v.id[i];
    }
  }
}

// Per-device set-up, once, with that device current: the device address of
// the scratch array and the scatter kernel's shared-memory limit.
std::mutex g_setup_mu;
int* g_hist_addr[64] = {nullptr};

int static_setup(int device, int** hist) {
  if (device < 0 || device >= 64) return PIC_EINVAL;
  std::lock_guard<std::mutex> lock(g_setup_mu);
  if (!g_hist_addr[device]) {
    void* ptr = nullptr;
    if (cudaGetSymbolAddress(&ptr, g_static_hist) != cudaSuccess || !ptr) return PIC_ECUDA;
    const int smem = kWarps * kMaxNz * (int)sizeof(int);
    if (cudaFuncSetAttribute(k_static_scatter, cudaFuncAttributeMaxDynamicSharedMemorySize, smem) !=
        cudaSuccess)
      return PIC_ECUDA;
    g_hist_addr[device] = static_cast<int*>(ptr);
  }
  *hist = g_hist_addr[device];
  return PIC_OK;
}

}  // namespace
}  // namespace pic

extern "C" int pic_sort_by_cell_static(const float* z, const float* vx, const float* vy,
                                       const float* vz, const uint32_t* id, int64_t n,
                                       int32_t n_cells, double gap_m, float* z_out,
                                       float* vx_out, float* vy_out, float* vz_out,
                                       uint32_t* id_out, void* cuda_stream) {
  using namespace pic;
  if (n < 0 || n_cells < 1 || n_cells > kMaxNz || !(gap_m > 0)) return PIC_EINVAL;
  if (n == 0) return PIC_OK;
  if (!z || !vx || !vy || !vz || !id || !z_out || !vx_out || !vy_out || !vz_out || !id_out)
    return PIC_EINVAL;
  // histogram entries and output positions are 32-bit
  if (n > (int64_t)INT32_MAX) return PIC_ECAPACITY;
  const long long nch = (n + kChunk - 1) / kChunk;
  if ((long long)n_cells * nch > kStaticHistInts) return PIC_ECAPACITY;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return PIC_ECUDA;
  View v;
  int rc = static_setup(dev, &v.hist);
  if (rc != PIC_OK) return rc;
  v.z = z; v.vx = vx; v.vy = vy; v.vz = vz; v.id = id;
  v.zo = z_out; v.vxo = vx_out; v.vyo = vy_out; v.vzo = vz_out; v.ido = id_out;
  v.n = n;
  v.nch = (int)nch;
  v.Nz = n_cells;
  v.inv_dz = (float)((double)n_cells / gap_m);
  cudaStream_t s = (cudaStream_t)cuda_stream;
  k_static_hist<<<(unsigned)nch, kThreads, n_cells * sizeof(int), s>>>(v);
  k_static_scan<<<1, 1024, 0, s>>>(v);
  k_static_scatter<<<(unsigned)nch, kThreads, (size_t)kWarps * n_cells * sizeof(int), s>>>(v);
  return cudaGetLastError() == cudaSuccess ? PIC_OK : PIC_ECUDA;
}
