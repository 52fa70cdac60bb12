// Frame-parallel CBP, log-tanh form (Sec. IV-C, Steps 1-3), for codes with small lifting
// sizes (down to Z = 1: codes given as plain parity-check matrices).  One thread decodes one
// frame at a time through the whole sequential schedule -- checks r*Z + z in ascending
// order, a check's edges in ascending column order -- so no thread waits for another and
// the kernel has no barrier after its table loads.  The per-edge arithmetic is that of
// the lane-parallel kernel (cbp_sp.cu), operation for operation, so both match the oracle
// bit for bit.
//
// Every per-frame array lives in the workspace element-major with the frame slot
// innermost (slot = the thread's index in the grid), so the threads of a warp, which walk
// the same edges in step, touch consecutive words -- one coalesced line per element:
//   QP  (Q*_v, phi(|Q*_v|)) of the variables of weight >= 2 columns  [idx*Z + z][slot]
//   SV  the same for weight-1 columns, indexed by the check lane        [idx*Z + z][slot]
//   S   check-beliefs S_c, sign bit = sgn Omega_c                       [M][slot]
//   R   C2V messages                                                     [E][slot]
//   B   decision bits of the flushed posterior                           [words][slot]
// The edge records (SpEdge) are read from global memory through L1: the threads of a warp
// read the same record at the same time.
#include "cbp_kernel_common.cuh"

namespace cbp {
namespace {

constexpr int kFpChunk = 6;   // edges of a check whose loads are issued together
constexpr int kFpBlock = 8;   // variables / syndrome terms per batch of loads
constexpr int kFpThreads = 256;

__global__ void __launch_bounds__(kFpThreads) cbp_fp_kernel(const KParams p) {
  extern __shared__ __align__(16) unsigned char smem[];
  float4* s_tab = reinterpret_cast<float4*>(smem);
  int* s_rptr = reinterpret_cast<int*>(s_tab + kPhiSegments);
  uint2* s_col = reinterpret_cast<uint2*>(s_rptr + ((p.mb + 1 + 3) & ~3));
  const int tid = threadIdx.x;
  for (int i = tid; i < kPhiSegments; i += blockDim.x) s_tab[i] = p.phi_tab[i];
  for (int i = tid; i <= p.mb; i += blockDim.x) s_rptr[i] = p.rptr[i];
  for (int c = tid; c < p.nb; c += blockDim.x) {  // (last row | shift << 16, idx | self << 16)
    const ColEntry ce = p.cols[p.cptr[c + 1] - 1];
    const BaseEdge be = p.edges[ce.e];
    s_col[c] = make_uint2(uint32_t(ce.r) | (uint32_t(ce.s) << 16),
                          (be.pad & 0xffffu) | ((be.flags & kSelf) ? 0x10000u : 0u));
  }
  __syncthreads();
  const long long slots = p.fp_slots;
  const long long slot = static_cast<long long>(blockIdx.x) * blockDim.x + tid;
  if (slot >= slots) return;
  const int Z = p.Z, N = p.N, words = p.words;
  const float xlo = p.phi_xlo;
  const float4* tab = s_tab;
  const SpEdge* __restrict__ spe = p.spe;
  // element e of an array sits at base[e * slots]
  float2* QP = reinterpret_cast<float2*>(p.ws) + slot;
  float2* SV = reinterpret_cast<float2*>(p.ws + p.fp_off_sv) + slot;
  float* S = p.ws + p.fp_off_s + slot;
  float* R = p.ws + p.fp_off_r + slot;
  uint32_t* B = reinterpret_cast<uint32_t*>(p.ws + p.fp_off_b) + slot;

  for (long long frame = slot; frame < p.batch; frame += slots) {
    // ---- Step 1, Eq. (s4e15): Q*_v = L_v (+0 turns -0 into +0)
    const float* src = p.llr + frame * N;
    bool bad = false;
    for (int c = 0; c < p.nb; ++c) {
      const uint2 ci = s_col[c];
      const int idx = ci.y & 0xffff;
      const bool self = ci.y & 0x10000u;
      const int sk = int(ci.x >> 16);
      for (int z = 0; z < Z; ++z) {  // a weight-1 column's state is indexed by its check lane
        const int v = self ? c * Z + mod_add(z + sk, Z) : c * Z + z;
        const float L = __fadd_rn(__ldg(src + v), 0.0f);
        bad |= non_finite(L);
        (self ? SV : QP)[static_cast<long long>(idx * Z + z) * slots] = make_float2(L, 0.0f);
      }
    }
    if (bad) atomicOr(p.status, kStatusNonFiniteLlr);

    for (int t = 1;; ++t) {
      // ---- Step 2: the checks in the sequential order
      for (int r = 0; r < p.mb; ++r) {
        const int k0 = s_rptr[r], k1 = s_rptr[r + 1];
        for (int z = 0; z < Z; ++z) {
          float Sacc = 0.0f;
          uint32_t sig = 0;
          for (int kb = k0; kb < k1; kb += kFpChunk) {
            float q[kFpChunk], ph[kFpChunk], sj[kFpChunk], ro[kFpChunk];
            int qoff[kFpChunk], roff[kFpChunk];
            uint32_t fl[kFpChunk];
#pragma unroll
            for (int j = 0; j < kFpChunk; ++j) {  // loads of the chunk
              const int k = kb + j;
              if (k < k1) {
                const SpEdge se = __ldg(spe + k);
                const int tq = static_cast<int>(se.w & 0xffffu), tj = static_cast<int>(se.w >> 16);
                const int uj = z >= tj ? Z : 0;
                fl[j] = se.x;
                qoff[j] = static_cast<int>(se.x & kSpMask) + z - (z >= tq ? Z : 0);
                roff[j] = static_cast<int>(se.z) + z - uj;
                const bool self = se.x & kSpSelf;
                const float2 qp = (self ? SV : QP)[static_cast<long long>(qoff[j]) * slots];
                q[j] = qp.x;
                ph[j] = qp.y;
                ro[j] = (!self && t > 1) ? R[static_cast<long long>(k * Z + z) * slots] : 0.0f;
                sj[j] = S[static_cast<long long>(static_cast<int>(se.y) + z - uj) * slots];
              }
            }
#pragma unroll
            for (int j = 0; j < kFpChunk; ++j) {  // the updates, in column order
              if (kb + j < k1) {
                const bool self = fl[j] & kSpSelf;
                // B2V, Eqs. (s4e18), (s4e13); a variable not visited before adds no C2V
                const float mag = phi_eval(fabsf(__fsub_rn(fabsf(sj[j]), ph[j])), xlo, tab);
                const float rb = __uint_as_float(
                    __float_as_uint(mag) |
                    ((__float_as_uint(sj[j]) ^ __float_as_uint(q[j])) & 0x80000000u));
                const bool first = (t == 1) && (fl[j] & kSpFirst);
                const float Rn = first ? 0.0f : rb;
                // V2C, Eqs. (s4e20), (s4e19); weight-1 column: c_j == c_i
                const float rold = self ? Rn : ro[j];
                const float qn = __fsub_rn(__fadd_rn(q[j], Rn), rold);
                // C2B, Eq. (s4e21) as a sum of phi; the sign bits fold into sig
                const float phn = phi_eval(fabsf(qn), xlo, tab);
                Sacc = __fadd_rn(Sacc, phn);
                sig ^= __float_as_uint(qn);
                if (self) {
                  SV[static_cast<long long>(qoff[j]) * slots] = make_float2(qn, phn);
                } else {
                  if (!first) R[static_cast<long long>(roff[j]) * slots] = Rn;  // Eq. (s4e22)
                  QP[static_cast<long long>(qoff[j]) * slots] = make_float2(qn, phn);
                }
              }
            }
          }
          // Eq. (s4e23); the sign bit carries sgn(Omega)
          S[static_cast<long long>(r * Z + z) * slots] =
              __uint_as_float(__float_as_uint(Sacc) | (sig & 0x80000000u));
        }
      }
      // ---- flushed posterior (Eq. s4e20 with the last check of v), decisions (Eq. s2e7);
      // the variables in blocks whose loads are issued together
      uint32_t word = 0;
      for (int vb = 0, cb = 0, pb = 0; vb < N; vb += kFpBlock) {
        float2 qp[kFpBlock];
        float sk[kFpBlock];
#pragma unroll
        for (int j = 0, c = cb, pz = pb; j < kFpBlock; ++j) {  // (c, pz): column, position
          if (vb + j < N) {
            const uint2 ci = s_col[c];
            const int idx = ci.y & 0xffff;
            const bool self = ci.y & 0x10000u;
            int zk = pz - int(ci.x >> 16);  // lane of v's last check
            zk = zk < 0 ? zk + Z : zk;
            // a weight-1 column's state is indexed by that lane, other columns' by position
            qp[j] = (self ? SV : QP)[static_cast<long long>(idx * Z + (self ? zk : pz)) * slots];
            sk[j] = S[static_cast<long long>(int(ci.x & 0xffff) * Z + zk) * slots];
            if (++pz == Z) {
              pz = 0;
              ++c;
            }
          }
          if (j == kFpBlock - 1) {
            cb = c;
            pb = pz;
          }
        }
#pragma unroll
        for (int j = 0; j < kFpBlock; ++j) {
          const int v = vb + j;
          if (v < N) {
            const float mag = phi_eval(fabsf(__fsub_rn(fabsf(sk[j]), qp[j].y)), xlo, tab);
            const uint32_t sg = (__float_as_uint(sk[j]) ^ __float_as_uint(qp[j].x)) & 0x80000000u;
            const float lb = __fadd_rn(qp[j].x, __uint_as_float(__float_as_uint(mag) | sg));
            if (p.soft) p.soft[frame * N + v] = lb;
            word |= static_cast<uint32_t>(lb < 0.0f) << (v & 31);
            if ((v & 31) == 31 || v == N - 1) {
              B[static_cast<long long>(v >> 5) * slots] = word;
              word = 0;
            }
          }
        }
      }
      // ---- syndrome; the scan stops at the first unsatisfied check
      bool ok = true;
      for (int r = 0; r < p.mb && ok; ++r) {
        const int k0 = s_rptr[r], k1 = s_rptr[r + 1];
        for (int z = 0; z < Z && ok; ++z) {
          uint32_t par = 0;
          for (int kb = k0; kb < k1; kb += kFpBlock) {
            uint32_t wv[kFpBlock];
            int sh[kFpBlock];
#pragma unroll
            for (int j = 0; j < kFpBlock; ++j)
              if (kb + j < k1) {
                const BaseEdge be = p.edges[kb + j];
                const int v = be.c * Z + mod_add(z + be.s, Z);
                wv[j] = B[static_cast<long long>(v >> 5) * slots];
                sh[j] = v & 31;
              }
#pragma unroll
            for (int j = 0; j < kFpBlock; ++j)
              if (kb + j < k1) par ^= wv[j] >> sh[j];
          }
          ok = (par & 1u) == 0;
        }
      }
      if ((ok && p.stop == CBP_STOP_SYNDROME) || t >= p.max_iter) {  // Step 3
        uint32_t* ho = p.hard + frame * words;
        for (int w = 0; w < words; ++w) ho[w] = B[static_cast<long long>(w) * slots];
        p.iters[frame] = ok ? t : -t;
        break;
      }
    }
  }
}

}  // namespace

void* fp_kernel_ptr() { return reinterpret_cast<void*>(&cbp_fp_kernel); }

int fp_threads() { return kFpThreads; }

}  // namespace cbp
