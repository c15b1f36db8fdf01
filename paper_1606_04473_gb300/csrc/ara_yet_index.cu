// Event-major index of a device YET (the layout is described with YetIndex in
// ara_internal.cuh).  The YET of Section IV-B is trial-major: each trial lists its event
// occurrences.  The adjoint's histograms are indexed by event, so the index lists, per event and
// block of trials, the trials in which it occurs.  Built by a counting sort on the device:
//   1. per (block, event): the number of occurrences (atomic counts);
//   2. per (block, group of 32 events): the longest of the group's 32 lists, rounded up to 8;
//   3. the groups' offsets in the entry array (an exclusive scan, on the host: the build is
//      synchronous, and the array is one 32-bit length per group and block);
//   4. every occurrence takes the next position of its list (atomic cursor) and stores its
//      trial's offset within the block.
// The order of the entries within a list depends on the order of the atomics; the counts that
// the adjoint takes from the lists do not.

#include <algorithm>
#include <vector>

#include "ara_internal.cuh"

namespace ara {

__global__ void __launch_bounds__(256)
k_yx_count(int64_t n_trials, const int64_t* __restrict__ off, int64_t n_events,
           const int32_t* __restrict__ ids, int64_t C, int64_t B, uint32_t* __restrict__ counts,
           uint32_t* __restrict__ err) {
  const int lane = threadIdx.x & 31;
  const int64_t w0 = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  uint32_t bad = 0;
  for (int64_t t = w0; t < n_trials; t += nw) {
    const int64_t beg = __ldg(off + t), end = __ldg(off + t + 1);
    if (!(0 <= beg && beg <= end && end <= n_events)) {
      bad |= DERR_OFFSETS;
      continue;
    }
    uint32_t* row = counts + (t / B) * C;
    for (int64_t i = beg + lane; i < end; i += 32) {
      const uint32_t e = (uint32_t)__ldcs(ids + i);
      if (e < (uint32_t)C) atomicAdd(row + e, 1u);
      else bad |= DERR_EVENT_RANGE;
    }
  }
  if (bad) atomicOr(err, bad);
}

// len[h][g] = the longest list of group g in block h, rounded up to a multiple of 8.
// total = n_blocks * groups * 32, a multiple of 32: every warp is wholly inside or outside.
__global__ void __launch_bounds__(256)
k_yx_len(int64_t total, int64_t C, int64_t G, const uint32_t* __restrict__ counts,
         uint32_t* __restrict__ len) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if ((i & ~(int64_t)31) >= total) return;
  const int64_t h = i / (G * 32), e = i % (G * 32);
  const uint32_t c = e < C ? counts[h * C + e] : 0u;
  const uint32_t m = __reduce_max_sync(0xffffffffu, c);
  if ((i & 31) == 0) len[i >> 5] = (m + 7u) & ~7u;
}

__global__ void __launch_bounds__(256)
k_yx_scatter(int64_t n_trials, const int64_t* __restrict__ off, int64_t n_events,
             const int32_t* __restrict__ ids, int64_t C, int64_t B, int64_t G,
             const int64_t* __restrict__ base, const uint32_t* __restrict__ len,
             uint32_t* __restrict__ cursor, uint16_t* __restrict__ ent, uint32_t* __restrict__ err) {
  const int lane = threadIdx.x & 31;
  const int64_t w0 = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  uint32_t bad = 0;
  for (int64_t t = w0; t < n_trials; t += nw) {
    const int64_t beg = __ldg(off + t), end = __ldg(off + t + 1);
    if (!(0 <= beg && beg <= end && end <= n_events)) continue;   // reported by the count
    const int64_t h = t / B;
    const uint16_t rel = (uint16_t)(t - h * B);
    for (int64_t i = beg + lane; i < end; i += 32) {
      const uint32_t e = (uint32_t)__ldcs(ids + i);
      if (e >= (uint32_t)C) continue;                              // reported by the count
      const int64_t hg = h * G + (e >> 5);
      const uint32_t k = atomicAdd(cursor + h * C + e, 1u);
      if (k < len[hg]) ent[base[hg] + (int64_t)(k >> 3) * 256 + (e & 31) * 8 + (k & 7)] = rel;
      else bad |= DERR_EVENT_RANGE;                                // the YET changed meanwhile
    }
  }
  if (bad) atomicOr(err, bad);
}

static void free_index(YetIndex* yx) {
  if (!yx) return;
  DeviceGuard g(yx->device);
  cudaFree(yx->d_ent);
  cudaFree(yx->d_base);
  cudaFree(yx->d_len);
}

}  // namespace ara

using namespace ara;

extern "C" ara_status ara_yet_index_create(ara_portfolio* pf_, int64_t n_trials,
                                           const int64_t* d_off, int64_t n_events,
                                           const int32_t* d_ids, void* stream,
                                           ara_yet_index** out) {
  Portfolio* pf = static_cast<Portfolio*>(pf_);
  if (!out) return ARA_EINVAL;
  *out = nullptr;
  if (!pf || n_trials < 1 || n_events < 0 || !d_off || (n_events > 0 && !d_ids)) return ARA_EINVAL;
  if (((uintptr_t)d_off & 7) || ((uintptr_t)d_ids & 3)) return ARA_EINVAL;
  if (pf->catalogue < 1 || pf->catalogue > (int64_t)UINT32_MAX) return ARA_EINVAL;
  DeviceGuard dg(pf->device);
  cudaStream_t s = (cudaStream_t)stream;
  const int64_t C = pf->catalogue, G = (C + 31) / 32;
  const int64_t H = (n_trials + YX_MAX_BLOCK - 1) / YX_MAX_BLOCK;
  const int64_t B = (n_trials + H - 1) / H;
  if (H > INT32_MAX) return ARA_ERANGE;
  ara_yet_index* yx = new ara_yet_index();
  yx->device = pf->device;
  yx->n_trials = n_trials;
  yx->n_events = n_events;
  yx->catalogue = C;
  yx->block = B;
  yx->n_blocks = (int32_t)H;
  yx->groups = G;
  uint32_t* d_cnt = nullptr;
  uint32_t* d_err = nullptr;
  auto fail = [&](ara_status e) {
    if (d_cnt) cudaFreeAsync(d_cnt, s);
    if (d_err) cudaFreeAsync(d_err, s);
    cudaStreamSynchronize(s);
    free_index(yx);
    delete yx;
    return e;
  };
  auto cuda_status = [](cudaError_t e) {
    return e == cudaErrorMemoryAllocation ? ARA_ENOMEM : ARA_ECUDA;
  };
  cudaError_t e;
  if ((e = dmalloc_async((void**)&d_cnt, sizeof(uint32_t) * (size_t)(H * C), s)) != cudaSuccess ||
      (e = dmalloc_async((void**)&d_err, sizeof(uint32_t), s)) != cudaSuccess ||
      (e = cudaMalloc((void**)&yx->d_len, sizeof(uint32_t) * (size_t)(H * G))) != cudaSuccess ||
      (e = cudaMalloc((void**)&yx->d_base, sizeof(int64_t) * (size_t)(H * G))) != cudaSuccess)
    return fail(cuda_status(e));
  const unsigned grid = (unsigned)std::max(1, pf->n_sms * 8);
  if ((e = cudaMemsetAsync(d_cnt, 0, sizeof(uint32_t) * (size_t)(H * C), s)) != cudaSuccess ||
      (e = cudaMemsetAsync(d_err, 0, sizeof(uint32_t), s)) != cudaSuccess)
    return fail(ARA_ECUDA);
  k_yx_count<<<grid, 256, 0, s>>>(n_trials, d_off, n_events, d_ids, C, B, d_cnt, d_err);
  const int64_t total = H * G * 32;
  k_yx_len<<<(unsigned)((total + 255) / 256), 256, 0, s>>>(total, C, G, d_cnt, yx->d_len);
  if (cudaGetLastError() != cudaSuccess) return fail(ARA_ECUDA);
  std::vector<uint32_t> len((size_t)(H * G));
  uint32_t h_err = 0;
  if (cudaMemcpyAsync(len.data(), yx->d_len, sizeof(uint32_t) * len.size(), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
      cudaMemcpyAsync(&h_err, d_err, sizeof(uint32_t), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
      cudaStreamSynchronize(s) != cudaSuccess)
    return fail(ARA_ECUDA);
  if (h_err) return fail(ARA_EDATA);
  std::vector<int64_t> base(len.size());
  int64_t n_ent = 0;
  for (size_t i = 0; i < len.size(); ++i) {
    base[i] = n_ent;
    n_ent += (int64_t)len[i] * 32;
  }
  yx->n_ent = n_ent;
  if ((e = cudaMalloc((void**)&yx->d_ent, sizeof(uint16_t) * (size_t)std::max<int64_t>(n_ent, 1))) != cudaSuccess)
    return fail(cuda_status(e));
  if (cudaMemcpyAsync(yx->d_base, base.data(), sizeof(int64_t) * base.size(), cudaMemcpyHostToDevice, s) != cudaSuccess ||
      cudaMemsetAsync(yx->d_ent, 0xC0, sizeof(uint16_t) * (size_t)n_ent, s) != cudaSuccess ||
      cudaMemsetAsync(d_cnt, 0, sizeof(uint32_t) * (size_t)(H * C), s) != cudaSuccess)
    return fail(ARA_ECUDA);
  static_assert(YX_PAD == 0xC0C0u, "the padding is the byte pattern 0xC0");
  k_yx_scatter<<<grid, 256, 0, s>>>(n_trials, d_off, n_events, d_ids, C, B, G, yx->d_base,
                                    yx->d_len, d_cnt, yx->d_ent, d_err);
  if (cudaGetLastError() != cudaSuccess) return fail(ARA_ECUDA);
  if (cudaMemcpyAsync(&h_err, d_err, sizeof(uint32_t), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
      cudaStreamSynchronize(s) != cudaSuccess)
    return fail(ARA_ECUDA);
  if (h_err) return fail(ARA_EDATA);
  cudaFreeAsync(d_cnt, s);
  cudaFreeAsync(d_err, s);
  d_cnt = nullptr;
  d_err = nullptr;
  if (cudaStreamSynchronize(s) != cudaSuccess) return fail(ARA_ECUDA);
  *out = yx;
  return ARA_OK;
}

extern "C" void ara_yet_index_destroy(ara_yet_index* yx) {
  if (!yx) return;
  free_index(yx);
  delete yx;
}
