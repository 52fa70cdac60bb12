// CBP, log-tanh form (Sec. IV-C, Steps 1-3): the main decoder kernel on sm_103a.
//
// Same frame-slot / Z-lane structure as the generic sequential kernel (one CTA holds
// F frames of Z lanes; the Z checks of a base row run in parallel, one barrier per
// row), with the per-frame state arranged for throughput:
//   shared    (Q*_v, phi(|Q*_v|)) pairs of the variables whose column has weight >= 2,
//             the check-beliefs S_c (sign bit = sgn Omega_c) when they fit, decision bits
//   workspace C2V messages R [base entry][lane]; (Q*, phi) of weight-1 columns, which
//             only their one check lane touches ([weight-1 column][lane]); S_c otherwise
// A base row is processed in chunks of CH edges: the loads of a chunk (Q*, phi, S of
// the predecessor check, R of the edge) are issued together, then the CH edge
// updates run with independent phi evaluations, in ascending column order.
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

template <bool CHKS, int CH>
__global__ void __launch_bounds__(1024, 1) cbp_sp_kernel(const KParams p) {
  extern __shared__ __align__(16) unsigned char smem[];
  const int Z = p.Z, N = p.N, M = p.M, words = p.words, F = p.F;
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
  uint2* s_col = reinterpret_cast<uint2*>(sp);  // per column: (last row | shift << 16, idx | self << 16)
  sp += sizeof(uint2) * ((p.nb + 1) & ~1);
  SlotState* s_slot = reinterpret_cast<SlotState*>(sp);
  sp += sizeof(SlotState) * ((F + 3) & ~3);
  float* s_frames = reinterpret_cast<float*>(sp);

  for (int i = tid; i < kPhiSegments; i += blockDim.x) s_tab[i] = p.phi_tab[i];
  for (int i = tid; i < p.nnzb; i += blockDim.x) s_e[i] = p.edges[i];
  for (int i = tid; i <= p.mb; i += blockDim.x) s_rptr[i] = p.rptr[i];
  for (int c = tid; c < p.nb; c += blockDim.x) {
    const ColEntry ce = p.cols[p.cptr[c + 1] - 1];
    const BaseEdge be = p.edges[ce.e];
    s_col[c] = make_uint2(uint32_t(ce.r) | (uint32_t(ce.s) << 16),
                          (be.pad & 0xffffu) | ((be.flags & kSelf) ? 0x10000u : 0u));
  }
  if (tid < F) {
    s_slot[tid].frame = blockIdx.x * F + tid;
    s_slot[tid].t = 0;
    s_slot[tid].unsat = 0;
  }
  // per frame, shared: QP float2 [ncomp*Z] | S [M] (CHKS) | bits [words]
  const int ncomp = p.ncomp;
  float* base = s_frames + static_cast<size_t>(lane ? f : 0) * p.sh_frame;
  float2* QP = reinterpret_cast<float2*>(base);
  float* nxt = base + 2 * static_cast<size_t>(ncomp) * Z;
  const long long g = static_cast<long long>(blockIdx.x) * F + (lane ? f : 0);
  float* wsl = p.ws + g * p.ws_slot;
  float* R = wsl;
  float2* SV = reinterpret_cast<float2*>(wsl + p.ws_off_sv);  // weight-1 columns
  float* S;
  if (CHKS) {
    S = nxt;
    nxt += (M + 3) & ~3;
  } else {
    S = wsl + p.ws_off_s;
  }
  uint32_t* bits = reinterpret_cast<uint32_t*>(nxt);
  const float4* tab = s_tab;
  const float xlo = p.phi_xlo;
  __syncthreads();

  for (;;) {
    const int frame = lane ? s_slot[f].frame : p.batch;
    const bool act = frame < p.batch;
    if (act && s_slot[f].t == 0) {  // Step 1, Eq. (s4e15): Q*_v = L_v
      const float* src = p.llr + static_cast<long long>(frame) * N;
      for (int c = 0; c < p.nb; ++c) {
        const uint32_t cinfo = s_col[c].y;
        const int idx = cinfo & 0xffff;
        if (cinfo & 0x10000u) {
          const int s = int(s_col[c].x >> 16);
          SV[idx * Z + z] = make_float2(__ldg(src + c * Z + mod_add(z + s, Z)), 0.0f);
        } else {
          QP[idx * Z + z] = make_float2(__ldg(src + c * Z + z), 0.0f);
        }
      }
    }
    if (!__syncthreads_or(act)) break;
    const int t = act ? s_slot[f].t + 1 : 0;

    for (int r = 0; r < p.mb; ++r) {
      if (act) {
        const int k0 = s_rptr[r], k1 = s_rptr[r + 1];
        float Sacc = 0.0f;
        uint32_t sig = 0;
        for (int kb = k0; kb < k1; kb += CH) {
          float q[CH], ph[CH], sj[CH], ro[CH];
#pragma unroll
          for (int j = 0; j < CH; ++j) {
            const int k = kb + j;
            if (k < k1) {
              const BaseEdge be = s_e[k];
              const int zv = mod_add(z + be.s, Z);
              const int idx = be.pad & 0xffff;
              float2 qp;
              if (be.flags & kSelf) qp = SV[idx * Z + z];
              else qp = QP[idx * Z + zv];
              q[j] = qp.x;
              ph[j] = qp.y;
              int zj = zv - be.ps;
              zj = zj < 0 ? zj + Z : zj;
              sj[j] = S[be.pr * Z + zj];
              ro[j] = (t > 1 && !(be.flags & kSelf)) ? R[k * Z + z] : 0.0f;
            }
          }
#pragma unroll
          for (int j = 0; j < CH; ++j) {
            const int k = kb + j;
            if (k < k1) {
              const BaseEdge be = s_e[k];
              const int zv = mod_add(z + be.s, Z);
              const bool self = be.flags & kSelf;
              float Rn = 0.0f;
              if (!(t == 1 && (be.flags & kFirst))) {
                // B2V, Eqs. (s4e18), (s4e13): exclude phi(|Q*|) from S of c_j
                const float mag = phi_eval(fabsf(__fsub_rn(fabsf(sj[j]), ph[j])), xlo, tab);
                Rn = (sign_bit(sj[j]) ^ (q[j] < 0.0f)) ? -mag : mag;
                if (!self) {                   // R_{c_j->v} <- R^new (Eq. s4e22)
                  int zj = zv - be.ps;
                  zj = zj < 0 ? zj + Z : zj;
                  R[be.pe * Z + zj] = Rn;
                }
              }
              const float rold = self ? Rn : ro[j];
              const float qn = __fsub_rn(__fadd_rn(q[j], Rn), rold);  // Eqs. (s4e20), (s4e19)
              const float phn = phi_eval(fabsf(qn), xlo, tab);        // C2B, Eq. (s4e21)
              Sacc = __fadd_rn(Sacc, phn);
              sig ^= (qn < 0.0f);
              const int idx = be.pad & 0xffff;
              if (self) SV[idx * Z + z] = make_float2(qn, phn);
              else QP[idx * Z + zv] = make_float2(qn, phn);
            }
          }
        }
        S[r * Z + z] = sig ? -Sacc : Sacc;     // Eq. (s4e23)
      }
      __syncthreads();
    }

    // ---- flushed posterior, hard decisions (Eq. s2e7)
    if (act)
      for (int w = z; w < words; w += Z) bits[w] = 0u;
    if (tid < F) s_slot[tid].unsat = 0;
    __syncthreads();
    {
      float* so = (act && p.soft) ? p.soft + static_cast<long long>(frame) * N : nullptr;
      for (int c = 0; c < p.nb; ++c) {
        const uint2 ci = s_col[c];
        const int idx = ci.y & 0xffff;
        const int sk = int(ci.x >> 16), rk = int(ci.x & 0xffff);
        int v = 0;
        bool neg = false;
        if (act) {
          float2 qp;
          float Sk;
          if (ci.y & 0x10000u) {  // weight-1 column: lane z owns its single check (rk, z)
            qp = SV[idx * Z + z];
            Sk = S[rk * Z + z];
            v = c * Z + mod_add(z + sk, Z);
          } else {
            qp = QP[idx * Z + z];
            int zk = z - sk;
            zk = zk < 0 ? zk + Z : zk;
            Sk = S[rk * Z + zk];
            v = c * Z + z;
          }
          const float mag = phi_eval(fabsf(__fsub_rn(fabsf(Sk), qp.y)), xlo, tab);
          const float lb = __fadd_rn(qp.x, (sign_bit(Sk) ^ (qp.x < 0.0f)) ? -mag : mag);
          neg = lb < 0.0f;
          if (so) so[v] = lb;
        }
        warp_or_bit(bits + (v >> 5), neg ? (1u << (v & 31)) : 0u, act);
      }
    }
    __syncthreads();
    // ---- syndrome; a frame stops scanning at its first unsatisfied check row
    if (act) {
      for (int r = 0; r < p.mb; ++r) {
        uint32_t pr = 0;
        for (int k = s_rptr[r]; k < s_rptr[r + 1]; ++k) {
          const BaseEdge be = s_e[k];
          const int v = be.c * Z + mod_add(z + be.s, Z);
          pr ^= bits[v >> 5] >> (v & 31);
        }
        if (pr & 1u) s_slot[f].unsat = 1;
        if (*static_cast<volatile int*>(&s_slot[f].unsat)) break;
      }
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

}  // namespace

void* sp_kernel_ptr(bool chk_shared) {
  return chk_shared ? reinterpret_cast<void*>(&cbp_sp_kernel<true, 4>)
                    : reinterpret_cast<void*>(&cbp_sp_kernel<false, 4>);
}

}  // namespace cbp
