// Sequential-schedule decoders on sm_103a: CBP normalized min-sum and the layered
// normalized min-sum comparator (CBP in log-tanh form has its own kernel, cbp_sp.cu).
//
// Parallel layout.  A CTA holds F frame slots of Z lanes each.  The checks of one
// base row r (m = r*Z + i, i = 0..Z-1) share no variable: every base column is a
// permutation of the Z variables of its block.  Processing a base row's Z checks in
// parallel therefore performs exactly the operations of the check-by-check order of
// Step 2 (Sec. IV-C), and one __syncthreads() per base row orders the rows.  Frames
// are independent; each slot decodes its own frame and, when that frame stops, loads
// the next one (slot g of the launch decodes frames g, g + slots, g + 2 slots, ...).
//
// Per frame slot:
//   shared:    Q*_v (CBP) or Lambda_v (LBP) (N), the CBP check state (min1 with the
//              sign of Omega, min2: 2M) when it fits, hard-decision bits (ceil(N/32) words)
//   workspace: the C2V messages R (E floats, [base entry][lane]), and the check
//              state when it does not fit in shared memory.
// The C2V message of edge (c_j, v) is produced when v is visited by the next check
// c_i holding it (B2V, Eq. s4e18) and consumed at c_j's own next visit (V2C, Eq. s4e19).
#include "cbp_internal.cuh"

namespace cbp {
namespace {

constexpr float kInf = __builtin_huge_valf();

struct SlotState {
  int frame;   // frame decoded by this slot (>= batch: idle)
  int t;       // sweeps completed (0: frame must be loaded)
  int unsat;   // some check unsatisfied after the current sweep
};

__device__ __forceinline__ int mod_add(int a, int Z) { return a >= Z ? a - Z : a; }
__device__ __forceinline__ uint32_t sign_bit(float x) { return __float_as_uint(x) >> 31; }

// ---------------------------------------------------------------------------
// Per-lane work of one check for one frame.
// ---------------------------------------------------------------------------
struct Ctx {
  int Z;
  int t;                       // current sweep (1-based)
  const BaseEdge* __restrict__ e;
  float* __restrict__ Q;       // Q*_v (CBP) or Lambda_v (LBP), shared
  float* __restrict__ C0;      // check state 0: signed min1 (CBP-NMS)
  float* __restrict__ C1;      // check state 1: min2 (CBP-NMS)
  float* __restrict__ R;       // C2V messages of this slot, global
  float alpha;
};

// CBP normalized min-sum, Eqs. (s4e18xx), (s4e21xx).
__device__ __forceinline__ void cbp_nms_check(const Ctx& x, int r, int k0, int k1, int z) {
  const int Z = x.Z;
  float m1 = kInf, m2 = kInf;
  uint32_t sig = 0;
  for (int k = k0; k < k1; ++k) {
    const BaseEdge be = x.e[k];
    const int zv = mod_add(z + be.s, Z);
    const int v = be.c * Z + zv;
    const bool self = be.flags & kSelf;
    const float Rold0 = (x.t > 1 && !self) ? x.R[k * Z + z] : 0.0f;
    const float q = x.Q[v];
    float Rn = 0.0f;
    if (!(x.t == 1 && (be.flags & kFirst))) {
      int zj = zv - be.ps;
      zj = zj < 0 ? zj + Z : zj;
      const float a1 = x.C0[be.pr * Z + zj];
      const float b1 = fabsf(a1);
      const float mag = (fabsf(q) == b1) ? x.C1[be.pr * Z + zj] : b1;
      const float rm = __fmul_rn(x.alpha, mag);
      Rn = (sign_bit(a1) ^ (q < 0.0f)) ? -rm : rm;
      x.R[be.pe * Z + zj] = Rn;
    }
    const float Rold = self ? Rn : Rold0;
    const float qn = __fsub_rn(__fadd_rn(q, Rn), Rold);
    const float a = fabsf(qn);
    if (a < m1) {
      m2 = m1;
      m1 = a;
    } else if (a < m2) {
      m2 = a;
    }
    sig ^= (qn < 0.0f);
    x.Q[v] = qn;
  }
  x.C0[r * Z + z] = sig ? -m1 : m1;
  x.C1[r * Z + z] = m2;
}

// Layered normalized min-sum, Eqs. (s2e10), (s2e12): two passes over the check,
// the V2C messages of the row held in registers between them.
__device__ __forceinline__ void lbp_nms_check(const Ctx& x, int r, int k0, int k1, int z) {
  const int Z = x.Z;
  const int d = k1 - k0;
  float qv[kMaxDeg];
  float m1 = kInf, m2 = kInf;
  int idx = -1;
  uint32_t sig = 0;
#pragma unroll
  for (int j = 0; j < kMaxDeg; ++j) {
    if (j < d) {
      const BaseEdge be = x.e[k0 + j];
      const int v = be.c * Z + mod_add(z + be.s, Z);
      const float Rold = x.t > 1 ? x.R[(k0 + j) * Z + z] : 0.0f;
      const float q = __fsub_rn(x.Q[v], Rold);
      qv[j] = q;
      const float a = fabsf(q);
      if (a < m1) {
        m2 = m1;
        m1 = a;
        idx = j;
      } else if (a < m2) {
        m2 = a;
      }
      sig ^= (q < 0.0f);
    }
  }
  const float r1 = __fmul_rn(x.alpha, m1), r2 = __fmul_rn(x.alpha, m2);
#pragma unroll
  for (int j = 0; j < kMaxDeg; ++j) {
    if (j < d) {
      const BaseEdge be = x.e[k0 + j];
      const int v = be.c * Z + mod_add(z + be.s, Z);
      const float rm = (j == idx) ? r2 : r1;
      const float Rn = (sig ^ (qv[j] < 0.0f)) ? -rm : rm;
      x.R[(k0 + j) * Z + z] = Rn;
      x.Q[v] = __fadd_rn(qv[j], Rn);
    }
  }
  (void)r;
}

// Flushed posterior of variable v (CBP min-sum), a read-only evaluation of Eq. (s4e20)
// with the last check of the sweep holding v as c_j.
__device__ __forceinline__ float cbp_flush(const Ctx& x, int v, int ci) {
  const float q = x.Q[v];
  const float a1 = x.C0[ci];
  const float b1 = fabsf(a1);
  const float mag = (fabsf(q) == b1) ? x.C1[ci] : b1;
  const float rm = __fmul_rn(x.alpha, mag);
  return __fadd_rn(q, (sign_bit(a1) ^ (q < 0.0f)) ? -rm : rm);
}

// ---------------------------------------------------------------------------
// The kernel.
// ---------------------------------------------------------------------------
template <int ALG, bool CHKS>
__global__ void __launch_bounds__(1024, 1) layered_kernel(const KParams p) {
  extern __shared__ __align__(16) unsigned char smem[];
  constexpr bool kLBP = (ALG == ALG_LBP_NMS);
  const int Z = p.Z, N = p.N, M = p.M, words = p.words, F = p.F;
  const int tid = threadIdx.x;
  const int f = tid / Z;
  const int z = tid - f * Z;
  const bool lane = f < F;

  // ---- shared-memory carve-up (must match shared_fixed_bytes / shared_frame_floats)
  unsigned char* sp = smem;
  BaseEdge* s_e = reinterpret_cast<BaseEdge*>(sp);
  sp += sizeof(BaseEdge) * p.nnzb;
  int* s_rptr = reinterpret_cast<int*>(sp);
  sp += sizeof(int) * ((p.mb + 1 + 3) & ~3);
  uint32_t* s_last = reinterpret_cast<uint32_t*>(sp);  // per column: (last row, shift)
  sp += sizeof(uint32_t) * ((p.nb + 3) & ~3);
  SlotState* s_slot = reinterpret_cast<SlotState*>(sp);
  sp += sizeof(SlotState) * ((F + 3) & ~3);
  float* s_frames = reinterpret_cast<float*>(sp);

  for (int i = tid; i < p.nnzb; i += blockDim.x) s_e[i] = p.edges[i];
  for (int i = tid; i <= p.mb; i += blockDim.x) s_rptr[i] = p.rptr[i];
  for (int c = tid; c < p.nb; c += blockDim.x) {
    const ColEntry ce = p.cols[p.cptr[c + 1] - 1];   // last row of column c
    s_last[c] = (uint32_t(ce.r) << 16) | ce.s;
  }
  if (tid < F) {
    s_slot[tid].frame = blockIdx.x * F + tid;
    s_slot[tid].t = 0;
    s_slot[tid].unsat = 0;
  }

  // per-frame shared arrays: Q [N] | C0 [M] | C1 [M] (CBP-NMS, CHKS) | bits [words]
  const int Npad = (N + 3) & ~3, Mpad = (M + 3) & ~3;
  float* base = s_frames + static_cast<size_t>(lane ? f : 0) * p.sh_frame;
  Ctx x;
  x.Z = Z;
  x.e = s_e;
  x.alpha = p.alpha;
  x.Q = base;
  float* nxt = base + Npad;
  const long long g = static_cast<long long>(blockIdx.x) * F + (lane ? f : 0);
  float* wsl = p.ws + g * p.ws_slot;
  x.R = wsl;
  x.C0 = x.C1 = nullptr;
  if (!kLBP) {
    if (CHKS) {
      x.C0 = nxt;
      x.C1 = nxt + Mpad;
      nxt += 2 * Mpad;
    } else {
      x.C0 = wsl + p.E;
      x.C1 = wsl + p.E + M;
    }
  }
  uint32_t* bits = reinterpret_cast<uint32_t*>(nxt);
  __syncthreads();

  const bool vec4 = (N & 3) == 0;
  for (;;) {
    // ---- load new frames into idle slots (Step 1: Q*_v = L_v, Eq. s4e15)
    const int frame = lane ? s_slot[f].frame : p.batch;
    const bool act = frame < p.batch;
    if (act && s_slot[f].t == 0) {
      const float* src = p.llr + static_cast<long long>(frame) * N;
      if (vec4) {
        const float4* s4 = reinterpret_cast<const float4*>(src);
        float4* d4 = reinterpret_cast<float4*>(x.Q);
        for (int i = z; i < (N >> 2); i += Z) d4[i] = __ldg(s4 + i);
      } else {
        for (int i = z; i < N; i += Z) x.Q[i] = __ldg(src + i);
      }
    }
    if (!__syncthreads_or(act)) break;
    x.t = act ? s_slot[f].t + 1 : 0;

    // ---- one sweep: base rows in order, the Z checks of a row in parallel
    for (int r = 0; r < p.mb; ++r) {
      if (act) {
        const int k0 = s_rptr[r], k1 = s_rptr[r + 1];
        if (ALG == ALG_CBP_NMS) cbp_nms_check(x, r, k0, k1, z);
        else lbp_nms_check(x, r, k0, k1, z);
      }
      __syncthreads();
    }

    // ---- hard decisions (Eq. s2e7) on the flushed posterior
    if (act)
      for (int w = z; w < words; w += Z) bits[w] = 0u;
    if (tid < F) s_slot[tid].unsat = 0;
    __syncthreads();
    if (act) {
      float* so = p.soft ? p.soft + static_cast<long long>(frame) * N : nullptr;
      for (int c = 0; c < p.nb; ++c) {
        const int v = c * Z + z;
        float lb;
        if (kLBP) {
          lb = x.Q[v];
        } else {
          const uint32_t l = s_last[c];
          int zk = z - int(l & 0xffffu);
          zk = zk < 0 ? zk + Z : zk;
          lb = cbp_flush(x, v, int(l >> 16) * Z + zk);
        }
        if (lb < 0.0f) atomicOr(bits + (v >> 5), 1u << (v & 31));
        if (so) so[v] = lb;
      }
    }
    __syncthreads();
    // ---- syndrome of check (r, z) for every base row
    if (act) {
      uint32_t par = 0;
      for (int r = 0; r < p.mb; ++r) {
        uint32_t pr = 0;
        for (int k = s_rptr[r]; k < s_rptr[r + 1]; ++k) {
          const BaseEdge be = s_e[k];
          const int v = be.c * Z + mod_add(z + be.s, Z);
          pr ^= bits[v >> 5] >> (v & 31);
        }
        par |= pr & 1u;
      }
      if (par) s_slot[f].unsat = 1;
    }
    __syncthreads();
    // ---- stop test and outputs
    bool done = false;
    if (act) {
      const bool ok = s_slot[f].unsat == 0;
      done = (ok && p.stop == CBP_STOP_SYNDROME) || x.t >= p.max_iter;
      if (done) {
        uint32_t* ho = p.hard + static_cast<long long>(frame) * words;
        for (int w = z; w < words; w += Z) ho[w] = bits[w];
        if (z == 0) p.iters[frame] = ok ? x.t : -x.t;
      }
    }
    __syncthreads();
    if (act && z == 0) {
      if (done) {
        s_slot[f].frame = frame + p.slots;
        s_slot[f].t = 0;
      } else {
        s_slot[f].t = x.t;
      }
    }
    __syncthreads();
  }
}

template <int ALG, bool CHKS>
void* kernel_ptr() {
  return reinterpret_cast<void*>(&layered_kernel<ALG, CHKS>);
}

}  // namespace

static void* select_kernel(const Variant& v) {
  switch (v.alg) {
    case ALG_CBP_SP: return sp_kernel_ptr(v.chk_shared);
    case ALG_CBP_NMS:
      return v.chk_shared ? kernel_ptr<ALG_CBP_NMS, true>() : kernel_ptr<ALG_CBP_NMS, false>();
    case ALG_LBP_NMS: return kernel_ptr<ALG_LBP_NMS, true>();
    case ALG_FBP_SP: return flood_kernel_ptr();
  }
  return nullptr;
}

cudaError_t decoder_func_attrs(const Variant& v, cudaFuncAttributes* a) {
  return cudaFuncGetAttributes(a, select_kernel(v));
}

cudaError_t decoder_set_smem(const Variant& v, int bytes) {
  return cudaFuncSetAttribute(select_kernel(v), cudaFuncAttributeMaxDynamicSharedMemorySize,
                              bytes);
}

cudaError_t decoder_occupancy(const Variant& v, int threads, size_t smem, int* ctas) {
  return cudaOccupancyMaxActiveBlocksPerMultiprocessor(ctas, select_kernel(v), threads, smem);
}

cudaError_t launch_decoder(const Variant& v, const KParams& p, int grid, int threads,
                           size_t smem, cudaStream_t st) {
  void* fn = select_kernel(v);
  void* args[] = {const_cast<KParams*>(&p)};
  return cudaLaunchKernel(fn, dim3(grid), dim3(threads), args, smem, st);
}

}  // namespace cbp
