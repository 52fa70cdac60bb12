// Device helpers shared by the sequential-schedule decoder kernels.
#pragma once

#include "cbp_internal.cuh"

namespace cbp {
namespace {

struct SlotState {
  int frame, t, unsat;
};

__device__ __forceinline__ int mod_add(int a, int Z) { return a >= Z ? a - Z : a; }
__device__ __forceinline__ uint32_t sign_bit(float x) { return __float_as_uint(x) >> 31; }

// OR `bit` into the shared word `word`, one atomic per distinct word in the warp (the
// lanes of a warp may belong to different frames, so words are matched by address).
__device__ __forceinline__ void warp_or_bit(uint32_t* word, uint32_t bit, bool active) {
  const unsigned act = __ballot_sync(0xffffffffu, active);
  if (!active) return;
  const unsigned grp = __match_any_sync(act, reinterpret_cast<unsigned long long>(word));
  const uint32_t val = __reduce_or_sync(grp, bit);
  if ((threadIdx.x & 31) == __ffs(grp) - 1 && val) atomicOr(word, val);
}

// Bulk prefetch of [a, b) into L2, shrunk to whole 16-byte units inside the range.
__device__ __forceinline__ void prefetch_l2(const float* a, const float* b) {
  const uintptr_t lo = (reinterpret_cast<uintptr_t>(a) + 15) & ~uintptr_t(15);
  const uintptr_t hi = reinterpret_cast<uintptr_t>(b) & ~uintptr_t(15);
  if (hi > lo)
    asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(lo),
                 "r"(static_cast<uint32_t>(hi - lo))
                 : "memory");
}

// Barrier over one team of lane groups (named barrier `id`, `n` threads; id 0 with
// n = blockDim.x is the whole CTA).  Teams run their sweeps independently, so one
// team's memory waits overlap another team's arithmetic.
__device__ __forceinline__ void team_sync(int id, int n) {
  asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(n) : "memory");
}
__device__ __forceinline__ bool team_sync_or(int id, int n, bool pred) {
  int r;
  asm volatile(
      "{\n\t.reg .pred p, q;\n\t"
      "setp.ne.u32 p, %1, 0;\n\t"
      "bar.red.or.pred q, %2, %3, p;\n\t"
      "selp.u32 %0, 1, 0, q;\n\t}"
      : "=r"(r)
      : "r"(static_cast<int>(pred)), "r"(id), "r"(n)
      : "memory");
  return r != 0;
}

}  // namespace
}  // namespace cbp
