// Random-gather throughput probe (a measurement tool built next to liblp.so;
// not part of the solver).  The iteration kernels' operand reads are random
// 8-byte gathers from an L2-resident vector; this probe measures the rate at
// which the GPU serves such gathers with nothing else in flight:
//   global:  __ldg gathers from a vector of M doubles (all blocks resident);
//   cluster: gathers from the vector split over the distributed shared memory
//            of 8-block clusters (each block holds M/8 doubles);
//   local:   gathers from a block's own shared memory (reference);
//   sliced:  the iteration kernels' access pattern in its simplest form --
//            one warp per slice of 32 columns, every column 10 elements,
//            int32 indices and FP64 values streamed (ld.global.cs) from a
//            126 MB matrix, one gather from a 1.6 MB vector per element, with
//            no epilogue, and with the column pass's per-column traffic (five
//            FP64 operands read, three written).
// Indices come from a per-thread linear congruential sequence (global,
// cluster) or a hash of the element number (sliced) reduced modulo the
// vector length, so every access is in bounds.  Prints one JSON line.
#include <cooperative_groups.h>

#include <cstdint>
#include <cstdio>

namespace cg = cooperative_groups;

namespace {

constexpr int kCS = 8;
constexpr int kChunk = 25000;  // doubles per block in the cluster variants (200 KB)
constexpr int kClusterM = kCS * kChunk;
constexpr int kIters = 512;    // gathers per thread

__device__ __forceinline__ uint32_t lcg(uint32_t &s) {
  s = s * 1664525u + 1013904223u;
  return s;
}

__global__ void gather_global(const double *__restrict__ y, uint32_t m, double *out) {
  uint32_t s = blockIdx.x * blockDim.x + threadIdx.x + 12345u;
  double acc = 0.0;
  for (int i = 0; i < kIters; i += 4) {
    const uint32_t a = lcg(s) % m, b = lcg(s) % m, c = lcg(s) % m, d = lcg(s) % m;
    acc += __ldg(y + a) + __ldg(y + b) + __ldg(y + c) + __ldg(y + d);
  }
  out[blockIdx.x * blockDim.x + threadIdx.x] = acc;
}

__global__ void __cluster_dims__(kCS, 1, 1) __launch_bounds__(1024)
gather_cluster(const double *__restrict__ y, double *out, int local_only) {
  extern __shared__ double buf[];
  cg::cluster_group cl = cg::this_cluster();
  const int rank = (int)cl.block_rank();
  for (int j = threadIdx.x; j < kChunk; j += blockDim.x) buf[j] = y[rank * kChunk + j];
  cl.sync();
  const double *base[kCS];
#pragma unroll
  for (int r = 0; r < kCS; ++r) base[r] = cl.map_shared_rank(buf, r);
  uint32_t s = blockIdx.x * blockDim.x + threadIdx.x + 12345u;
  double acc = 0.0;
  for (int i = 0; i < kIters; i += 4) {
    double v[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const uint32_t idx = lcg(s) % (local_only ? (uint32_t)kChunk : (uint32_t)kClusterM);
      const uint32_t r = local_only ? (uint32_t)rank : idx / kChunk;
      v[q] = local_only ? buf[idx] : base[r][idx - r * kChunk];
    }
    acc += v[0] + v[1] + v[2] + v[3];
  }
  out[blockIdx.x * blockDim.x + threadIdx.x] = acc;
  cl.sync();  // no block leaves while another may read its memory
}

// Slices of 32 columns with kSliceSteps elements each; element s of the
// slice's lane l sits at 32 * (kSliceSteps * slice + s) + l.
constexpr int kSliceSteps = 10;
constexpr int kSliceCols = 1 << 20;
constexpr uint32_t kSliceRows = 200000;

__global__ void slice_fill(int32_t *idx, double *val, int64_t nnz) {
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < nnz;
       k += (int64_t)gridDim.x * blockDim.x) {
    uint32_t h = (uint32_t)k * 2654435761u;
    h ^= h >> 15;
    h *= 2246822519u;
    h ^= h >> 13;
    idx[k] = (int32_t)(h % kSliceRows);
    val[k] = 1.0 + (double)(h & 7) * 0.125;
  }
}

// Two elements per lane in flight: index/value loads, then gathers, then FMAs.
template <bool EPI>
__global__ void __launch_bounds__(256) slice_spmv(const int32_t *__restrict__ idx,
                                                  const double *__restrict__ val,
                                                  const double *__restrict__ y,
                                                  const double *__restrict__ in,
                                                  double *__restrict__ out) {
  const int lane = threadIdx.x & 31;
  const int w = (int)((blockIdx.x * blockDim.x + threadIdx.x) >> 5);
  if (w >= kSliceCols / 32) return;
  const int64_t col = (int64_t)w * 32 + lane;
  double p[5] = {0, 0, 0, 0, 0};
  if (EPI) {
#pragma unroll
    for (int q = 0; q < 5; ++q) p[q] = __ldcs(in + (int64_t)q * kSliceCols + col);
  }
  const int64_t base = (int64_t)w * 32 * kSliceSteps + lane;
  double acc = -p[0];
  for (int t = 0; t < kSliceSteps; t += 2) {
    const int32_t j0 = __ldcs(idx + base + 32 * t), j1 = __ldcs(idx + base + 32 * (t + 1));
    const double c0 = __ldcs(val + base + 32 * t), c1 = __ldcs(val + base + 32 * (t + 1));
    const double g0 = __ldg(y + j0), g1 = __ldg(y + j1);
    acc = fma(c0, g0, acc);
    acc = fma(c1, g1, acc);
  }
  if (EPI) {
    const double xn = fmin(fmax(p[3] + 0.1 * acc, p[1]), p[2]);
    out[col] = xn;
    out[kSliceCols + col] = 2.0 * xn - p[3];
    out[2 * (int64_t)kSliceCols + col] = p[4] + (xn - p[4]) * 0.5;
  } else {
    out[col] = acc;
  }
}

}  // namespace

int main() {
  int nsm = 0;
  if (cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, 0) != cudaSuccess) return 1;
  const uint32_t big = 1000000;
  double *y = nullptr, *out = nullptr;
  if (cudaMalloc(&y, sizeof(double) * big) != cudaSuccess) return 1;
  if (cudaMalloc(&out, sizeof(double) * (size_t)nsm * 2048) != cudaSuccess) return 1;
  cudaMemset(y, 0, sizeof(double) * big);
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  float ms = 0.0f;
  double g_small = 0, g_big = 0, g_cl = 0, g_loc = 0;
  int ncl = 0;
  for (uint32_t m : {(uint32_t)kClusterM, big}) {
    const int blocks = nsm * 8, threads = 256;
    gather_global<<<blocks, threads>>>(y, m, out);
    cudaEventRecord(e0);
    for (int r = 0; r < 10; ++r) gather_global<<<blocks, threads>>>(y, m, out);
    cudaEventRecord(e1);
    cudaEventSynchronize(e1);
    cudaEventElapsedTime(&ms, e0, e1);
    const double rate = 10.0 * blocks * threads * (double)kIters / (ms * 1e6);
    (m == big ? g_big : g_small) = rate;
  }
  const size_t smem = sizeof(double) * kChunk;
  cudaFuncSetAttribute(gather_cluster, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  cudaLaunchConfig_t cfg = {};
  cfg.blockDim = dim3(1024);
  cfg.dynamicSmemBytes = smem;
  cfg.gridDim = dim3(kCS);
  if (cudaOccupancyMaxActiveClusters(&ncl, gather_cluster, &cfg) != cudaSuccess) ncl = 0;
  cudaGetLastError();
  for (int lo = 0; lo < 2 && ncl > 0; ++lo) {
    const int blocks = ncl * kCS;
    gather_cluster<<<blocks, 1024, smem>>>(y, out, lo);
    cudaEventRecord(e0);
    for (int r = 0; r < 10; ++r) gather_cluster<<<blocks, 1024, smem>>>(y, out, lo);
    cudaEventRecord(e1);
    cudaEventSynchronize(e1);
    cudaEventElapsedTime(&ms, e0, e1);
    (lo ? g_loc : g_cl) = 10.0 * blocks * 1024.0 * kIters / (ms * 1e6);
  }
  cudaGetLastError();
  // sliced SpMV with and without the column pass's per-column traffic
  double g_sl = 0, g_sle = 0;
  const int64_t snnz = (int64_t)kSliceCols * kSliceSteps;
  int32_t *sidx = nullptr;
  double *sval = nullptr, *svec = nullptr;
  if (cudaMalloc(&sidx, sizeof(int32_t) * snnz) == cudaSuccess &&
      cudaMalloc(&sval, sizeof(double) * snnz) == cudaSuccess &&
      cudaMalloc(&svec, sizeof(double) * 8 * (size_t)kSliceCols) == cudaSuccess) {
    cudaMemset(svec, 0, sizeof(double) * 8 * (size_t)kSliceCols);
    slice_fill<<<nsm * 8, 256>>>(sidx, sval, snnz);
    const int blocks = kSliceCols / 256;  // one warp per slice of 32 columns
    for (int e = 0; e < 2; ++e) {
      auto run = [&] {
        if (e) slice_spmv<true><<<blocks, 256>>>(sidx, sval, y, svec, svec + 5 * (size_t)kSliceCols);
        else slice_spmv<false><<<blocks, 256>>>(sidx, sval, y, svec, svec + 5 * (size_t)kSliceCols);
      };
      run();
      cudaEventRecord(e0);
      for (int r = 0; r < 20; ++r) run();
      cudaEventRecord(e1);
      cudaEventSynchronize(e1);
      cudaEventElapsedTime(&ms, e0, e1);
      (e ? g_sle : g_sl) = 20.0 * (double)snnz / (ms * 1e6);
    }
  }
  const cudaError_t err = cudaGetLastError();
  printf("{\"global_1p6MB_ggathers_per_s\": %.2f, \"global_8MB_ggathers_per_s\": %.2f, "
         "\"cluster_dsmem_ggathers_per_s\": %.2f, \"local_smem_ggathers_per_s\": %.2f, "
         "\"cluster_blocks_resident\": %d, \"sliced_spmv_ggathers_per_s\": %.2f, "
         "\"sliced_spmv_epilogue_ggathers_per_s\": %.2f, \"error\": \"%s\"}\n",
         g_small, g_big, g_cl, g_loc, ncl * kCS, g_sl, g_sle, cudaGetErrorString(err));
  cudaFree(sidx);
  cudaFree(sval);
  cudaFree(svec);
  cudaFree(y);
  cudaFree(out);
  return err == cudaSuccess ? 0 : 1;
}
