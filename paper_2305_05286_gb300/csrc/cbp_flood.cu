// Flooding sum-product BP (FBP) comparator on sm_103a, the elementwise phi kernel and the
// one-thread kernel that reads and clears a code's device status word.
//
// Per iteration (Sec. II-A): every check computes its C2V messages from the V2C
// messages Q_{v->c} = Lambda_v - R_{c->v} of the previous posterior (Eq. s3e1) with the
// shared phi-sum of Eq. (s3e2); then every variable forms the posterior
// Lambda_v = L_v + sum_c R_{c->v} (Eq. s2e6) in ascending check order and decides
// (Eq. s2e7).  Same slot structure as the sequential decoders: F frames per CTA, Z
// lanes per frame, Lambda in shared memory, R in the workspace ([base entry][lane]).
#include "cbp_internal.cuh"

namespace cbp {
namespace {

struct SlotState {
  int frame, t, unsat;
};

__device__ __forceinline__ int mod_add(int a, int Z) { return a >= Z ? a - Z : a; }

// Eqs. (s3e1), (s3e2) for check (r, z): d <= D edges starting at base entry k0.
template <int D>
__device__ __forceinline__ void fbp_check(const BaseEdge* __restrict__ s_e, int k0, int d, int z,
                                          int Z, int t, const float* lam, float* R, float xlo,
                                          const float4* __restrict__ tab) {
  float ph[D];
  uint32_t neg = 0, sig = 0;
  float S = 0.0f;
#pragma unroll
  for (int j = 0; j < D; ++j) {
    if (j < d) {
      const BaseEdge be = s_e[k0 + j];
      const int v = be.c * Z + mod_add(z + be.s, Z);
      const float q = __fsub_rn(lam[v], t > 1 ? R[(k0 + j) * Z + z] : 0.0f);
      const uint32_t n = q < 0.0f;
      neg |= n << j;
      sig ^= n;
      ph[j] = phi_eval(fabsf(q), xlo, tab);
      S = __fadd_rn(S, ph[j]);
    }
  }
#pragma unroll
  for (int j = 0; j < D; ++j) {
    if (j < d) {
      const float mag = phi_eval(fabsf(__fsub_rn(S, ph[j])), xlo, tab);
      R[(k0 + j) * Z + z] = (sig ^ ((neg >> j) & 1u)) ? -mag : mag;
    }
  }
}

__global__ void __launch_bounds__(768, 1) flood_kernel(const KParams p) {
  extern __shared__ __align__(16) unsigned char smem[];
  const int Z = p.Z, N = p.N, words = p.words, F = p.F;
  const int tid = threadIdx.x;
  const int f = tid / Z;
  const int z = tid - f * Z;
  const bool lane = f < F;

  unsigned char* sp = smem;
  float4* s_tab = reinterpret_cast<float4*>(sp);
  sp += sizeof(float4) * kPhiSegments;
  BaseEdge* s_e = reinterpret_cast<BaseEdge*>(sp);
  sp += sizeof(BaseEdge) * p.nnzb;
  int* s_rptr = reinterpret_cast<int*>(sp);
  sp += sizeof(int) * ((p.mb + 1 + 3) & ~3);
  ColEntry* s_col = reinterpret_cast<ColEntry*>(sp);
  sp += sizeof(ColEntry) * ((p.nnzb + 1) & ~1);
  int* s_cptr = reinterpret_cast<int*>(sp);
  sp += sizeof(int) * ((p.nb + 1 + 3) & ~3);
  SlotState* s_slot = reinterpret_cast<SlotState*>(sp);
  sp += sizeof(SlotState) * ((F + 3) & ~3);
  float* s_frames = reinterpret_cast<float*>(sp);

  for (int i = tid; i < kPhiSegments; i += blockDim.x) s_tab[i] = p.phi_tab[i];
  for (int i = tid; i < p.nnzb; i += blockDim.x) {
    s_e[i] = p.edges[i];
    s_col[i] = p.cols[i];
  }
  for (int i = tid; i <= p.mb; i += blockDim.x) s_rptr[i] = p.rptr[i];
  for (int i = tid; i <= p.nb; i += blockDim.x) s_cptr[i] = p.cptr[i];
  if (tid < F) {
    s_slot[tid].frame = blockIdx.x * F + tid;
    s_slot[tid].t = 0;
    s_slot[tid].unsat = 0;
  }
  const int Npad = (N + 3) & ~3;
  float* lam = s_frames + static_cast<size_t>(lane ? f : 0) * p.sh_frame;
  uint32_t* bits = reinterpret_cast<uint32_t*>(lam + Npad);
  const long long g = static_cast<long long>(blockIdx.x) * F + (lane ? f : 0);
  float* R = p.ws + g * p.ws_slot;
  const float xlo = p.phi_xlo;
  __syncthreads();

  for (;;) {
    const int frame = lane ? s_slot[f].frame : p.batch;
    const bool act = frame < p.batch;
    const float* L = p.llr + static_cast<long long>(act ? frame : 0) * N;
    if (act && s_slot[f].t == 0) {    // R = 0, so Lambda = L + 0 (Eq. s2e6)
      bool bad = false;
      for (int i = z; i < N; i += Z) {
        lam[i] = __fadd_rn(__ldg(L + i), 0.0f);
        bad |= non_finite(lam[i]);
      }
      if (bad) atomicOr(p.status, kStatusNonFiniteLlr);
    }
    if (!__syncthreads_or(act)) break;
    const int t = act ? s_slot[f].t + 1 : 0;

    // ---- every check of the frame: Eqs. (s3e1), (s3e2)
    if (act) {
      for (int w = z; w < words; w += Z) bits[w] = 0u;
      for (int r = 0; r < p.mb; ++r) {
        const int k0 = s_rptr[r], d = s_rptr[r + 1] - k0;
        if (d <= 8) fbp_check<8>(s_e, k0, d, z, Z, t, lam, R, xlo, s_tab);
        else if (d <= 16) fbp_check<16>(s_e, k0, d, z, Z, t, lam, R, xlo, s_tab);
        else fbp_check<kMaxDeg>(s_e, k0, d, z, Z, t, lam, R, xlo, s_tab);
      }
    }
    if (tid < F) s_slot[tid].unsat = 0;
    __syncthreads();
    // ---- posterior, Eq. (s2e6), and hard decision, Eq. (s2e7)
    if (act) {
      float* so = p.soft ? p.soft + static_cast<long long>(frame) * N : nullptr;
      for (int c = 0; c < p.nb; ++c) {
        const int v = c * Z + z;
        float s = __ldg(L + v);
        for (int k = s_cptr[c]; k < s_cptr[c + 1]; ++k) {
          const ColEntry ce = s_col[k];
          int i = z - int(ce.s);
          i = i < 0 ? i + Z : i;
          s = __fadd_rn(s, R[int(ce.e) * Z + i]);
        }
        lam[v] = s;
        if (s < 0.0f) atomicOr(bits + (v >> 5), 1u << (v & 31));
        if (so) so[v] = s;
      }
    }
    __syncthreads();
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
    bool done = false;
    if (act) {
      const bool ok = s_slot[f].unsat == 0;
      done = (ok && p.stop == CBP_STOP_SYNDROME) || t >= p.max_iter;
      if (done) {
        uint32_t* ho = p.hard + static_cast<long long>(frame) * words;
        for (int w = z; w < words; w += Z) ho[w] = bits[w];
        if (z == 0) p.iters[frame] = ok ? t : -t;
      }
    }
    __syncthreads();
    if (act && z == 0) {
      if (done) {
        s_slot[f].frame = frame + p.slots;
        s_slot[f].t = 0;
      } else {
        s_slot[f].t = t;
      }
    }
    __syncthreads();
  }
}

template <bool DERIV>
__global__ void phi_kernel(const float* __restrict__ x, float* __restrict__ y, long long n,
                           const float4* __restrict__ tab, float xlo) {
  const long long stride = static_cast<long long>(gridDim.x) * blockDim.x;
  for (long long i = static_cast<long long>(blockIdx.x) * blockDim.x + threadIdx.x; i < n;
       i += stride)
    y[i] = DERIV ? phi_deriv(x[i], xlo, tab) : phi_eval(x[i], xlo, tab);
}

}  // namespace

void* flood_kernel_ptr() { return reinterpret_cast<void*>(&flood_kernel); }

namespace {
// Read and clear a code's status word in one atomic step: flags set by kernels still
// running on other streams are either returned now or kept for the next read.
__global__ void status_take_kernel(uint32_t* s) { s[1] = atomicExch(s, 0u); }
}  // namespace

cudaError_t launch_status_take(uint32_t* status, cudaStream_t st) {
  status_take_kernel<<<1, 1, 0, st>>>(status);
  return cudaGetLastError();
}

cudaError_t launch_phi(const float* x, float* y, long long n, const float4* tab, float xlo,
                       cudaStream_t st, bool deriv) {
  if (n <= 0) return cudaSuccess;
  long long blocks = (n + 255) / 256;
  if (blocks > 4096) blocks = 4096;
  if (deriv)
    phi_kernel<true><<<static_cast<int>(blocks), 256, 0, st>>>(x, y, n, tab, xlo);
  else
    phi_kernel<false><<<static_cast<int>(blocks), 256, 0, st>>>(x, y, n, tab, xlo);
  return cudaGetLastError();
}

}  // namespace cbp
