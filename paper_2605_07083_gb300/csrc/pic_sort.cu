// pic_sort.cu -- stable counting sort of every (instance, species) particle
// segment by cell, run every few steps so that the blocks of the push kernel
// see narrow cell ranges (short charge flushes, local shared-memory atomics).
//
// Four passes per sort, each a 2D grid (chunk of kSortChunk particles,
// segment):
//   1. per-chunk cell histogram            -> hist[g][cell][chunk]
//   2. one block per segment: exclusive scan of hist in (cell, chunk) order
//   3. scatter: each warp owns a contiguous sub-chunk; per-(warp, cell)
//      offsets in shared memory; __match_any_sync ranks equal cells inside a
//      warp, so the order of equal cells is the original order (stable)
//   4. copy the sorted scratch arrays back
// The cell of a particle is the fixed-point deposit's cell rule.
#include "pic_internal.cuh"

namespace pic {

constexpr int kSortChunk = 8192;
constexpr int kSortThreads = 256;
constexpr int kSortWarps = kSortThreads / 32;

__device__ __forceinline__ int seg_nz(const DevState& st, int g) { return st.ic[g / 3].Nz; }

__device__ __forceinline__ int seg_chunks_cap(const DevState& st, int g) {
  return (st.seg_cap[g] + kSortChunk - 1) / kSortChunk;
}

__global__ void __launch_bounds__(kSortThreads) k_sort_hist(DevState st) {
  extern __shared__ int hs[];
  const int g = blockIdx.y, c = blockIdx.x;
  const int N = st.seg_count[g];
  const int nch = (N + kSortChunk - 1) / kSortChunk;
  if (c >= nch) return;
  const InstConst& ic = st.ic[g / 3];
  const int Nz = ic.Nz;
  for (int j = threadIdx.x; j < Nz; j += blockDim.x) hs[j] = 0;
  __syncthreads();
  const long long off = st.seg_off[g];
  const int i0 = c * kSortChunk, i1 = min(N, i0 + kSortChunk);
  const float inv_dz = ic.inv_dz_f;
  for (int i = i0 + threadIdx.x; i < i1; i += blockDim.x) {
    int j;
    float f;
    cell_of(st.z[off + i], inv_dz, Nz, j, f);
    atomicAdd(&hs[j], 1);
  }
  __syncthreads();
  const int nchc = seg_chunks_cap(st, g);
  int* h = st.sort_hist + st.sort_hoff[g];
  for (int j = threadIdx.x; j < Nz; j += blockDim.x) h[(long long)j * nchc + c] = hs[j];
}

__global__ void __launch_bounds__(1024) k_sort_scan(DevState st) {
  __shared__ int ws[32];
  const int g = blockIdx.x;
  const int N = st.seg_count[g];
  const int nch = (N + kSortChunk - 1) / kSortChunk;
  if (nch == 0) return;
  const int nchc = seg_chunks_cap(st, g);
  const int Nz = seg_nz(st, g);
  int* h = st.sort_hist + st.sort_hoff[g];
  // entries (cell j, chunk c < nch) in cell-major order; chunks >= nch are unused
  const long long n = (long long)Nz * nch;
  int carry = 0;
  for (long long base = 0; base < n; base += blockDim.x) {
    const long long k = base + threadIdx.x;
    int v = 0;
    long long addr = 0;
    if (k < n) {
      const long long j = k / nch, c = k - j * nch;
      addr = j * nchc + c;
      v = h[addr];
    }
    int tot;
    const int ex = block_exclusive_scan<int>(v, &tot, ws);
    if (k < n) h[addr] = carry + ex;
    carry += tot;
  }
}

__global__ void __launch_bounds__(kSortThreads) k_sort_scatter(DevState st) {
  extern __shared__ int woff[];               // [kSortWarps][Nz]
  const int g = blockIdx.y, c = blockIdx.x;
  const int N = st.seg_count[g];
  const int nch = (N + kSortChunk - 1) / kSortChunk;
  if (c >= nch) return;
  const InstConst& ic = st.ic[g / 3];
  const int Nz = ic.Nz;
  const float inv_dz = ic.inv_dz_f;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const long long off = st.seg_off[g];
  const int i0 = c * kSortChunk, i1 = min(N, i0 + kSortChunk);
  const int per = (kSortChunk / kSortWarps);
  const int w0 = i0 + warp * per, w1 = min(i1, w0 + per);
  for (int k = threadIdx.x; k < kSortWarps * Nz; k += blockDim.x) woff[k] = 0;
  __syncthreads();
  int* my = woff + warp * Nz;
  for (int i = w0 + lane; i < w1; i += 32) {
    int j;
    float f;
    cell_of(st.z[off + i], inv_dz, Nz, j, f);
    atomicAdd(&my[j], 1);
  }
  __syncthreads();
  const int nchc = seg_chunks_cap(st, g);
  const int* h = st.sort_hist + st.sort_hoff[g];
  for (int j = threadIdx.x; j < Nz; j += blockDim.x) {
    int run = h[(long long)j * nchc + c];
    for (int w = 0; w < kSortWarps; ++w) {
      const int cnt = woff[w * Nz + j];
      woff[w * Nz + j] = run;
      run += cnt;
    }
  }
  __syncthreads();
  const unsigned lt = (1u << lane) - 1u;
  for (int base = w0; base < w1; base += 32) {
    const int i = base + lane;
    const bool act = i < w1;
    const unsigned am = __ballot_sync(0xffffffffu, act);
    int j = -1;
    if (act) {
      float f;
      cell_of(st.z[off + i], inv_dz, Nz, j, f);
    }
    const unsigned peers = __match_any_sync(0xffffffffu, j) & am;
    int pos = 0;
    if (act) pos = my[j] + __popc(peers & lt);
    __syncwarp();
    if (act && (peers & lt) == 0u) my[j] += __popc(peers);
    __syncwarp();
    if (act) {
      st.z2[off + pos] = st.z[off + i];
      st.vx2[off + pos] = st.vx[off + i];
      st.vy2[off + pos] = st.vy[off + i];
      st.vz2[off + pos] = st.vz[off + i];
      st.id2[off + pos] = st.id[off + i];
    }
  }
}

__global__ void __launch_bounds__(kSortThreads) k_sort_copy(DevState st) {
  const int g = blockIdx.y, c = blockIdx.x;
  const int N = st.seg_count[g];
  const int i0 = c * kSortChunk, i1 = min(N, i0 + kSortChunk);
  const long long off = st.seg_off[g];
  for (int i = i0 + threadIdx.x; i < i1; i += blockDim.x) {
    st.z[off + i] = st.z2[off + i];
    st.vx[off + i] = st.vx2[off + i];
    st.vy[off + i] = st.vy2[off + i];
    st.vz[off + i] = st.vz2[off + i];
    st.id[off + i] = st.id2[off + i];
  }
}

size_t sort_hist_ints(const int32_t* seg_cap, const int* seg_nz, int n_seg, int64_t* hoff) {
  size_t tot = 0;
  for (int g = 0; g < n_seg; ++g) {
    hoff[g] = (int64_t)tot;
    tot += (size_t)seg_nz[g] * (size_t)((seg_cap[g] + kSortChunk - 1) / kSortChunk);
  }
  return tot;
}

int sort_max_chunks(const int32_t* seg_cap, int n_seg) {
  int m = 1;
  for (int g = 0; g < n_seg; ++g) m = max(m, (seg_cap[g] + kSortChunk - 1) / kSortChunk);
  return m;
}

size_t sort_scatter_smem(int max_nz) { return (size_t)kSortWarps * max_nz * sizeof(int); }

// raise the kernels' dynamic shared-memory limit to the opt-in maximum less
// their static shared memory
cudaError_t sort_prepare(int optin) {
  const void* fns[] = {(const void*)k_sort_scatter, (const void*)k_sort_hist};
  for (const void* f : fns) {
    cudaFuncAttributes a;
    cudaError_t e = cudaFuncGetAttributes(&a, f);
    if (e == cudaSuccess)
      e = cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize,
                               optin - (int)a.sharedSizeBytes);
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

void sort_launch(const DevState& st, int max_chunks, int max_nz, cudaStream_t s) {
  const dim3 grid(max_chunks, st.n_seg);
  k_sort_hist<<<grid, kSortThreads, max_nz * sizeof(int), s>>>(st);
  k_sort_scan<<<st.n_seg, 1024, 0, s>>>(st);
  k_sort_scatter<<<grid, kSortThreads, sort_scatter_smem(max_nz), s>>>(st);
  k_sort_copy<<<grid, kSortThreads, 0, s>>>(st);
}

}  // namespace pic
