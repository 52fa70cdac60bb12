// Normalized min-sum decoders on sm_103a: CBP min-sum (Eqs. s4e18xx, s4e21xx) and the
// layered normalized min-sum comparator (Eqs. s2e10, s2e12).
//
// Same frame-slot / team structure as the CBP log-tanh kernel (cbp_sp.cu): lane z of
// a lane group owns check r*Z + z of every base row, the Z checks of a row run in
// parallel, teams of whole warps synchronise on their own named barrier per row.
//
// Neither decoder stores per-edge C2V messages.  A check keeps its state
//   min1 of |Q| (its sign bit carries sgn Omega), min2, the position of min1 among the
//   check's edges, one sign bit per edge (sgn of the V2C message folded in)
// and the C2V message it sent to its j-th variable is rebuilt from that state as
// alpha * (j == argmin ? min2 : min1) with sign sgn(Omega) ^ sign_j: the very value
// the decoder computed when the message was first formed (a tie between equal minima
// gives min2 == min1, so position and value comparisons agree).
//   CBP min-sum: shared     Q*_v of weight >= 2 columns; (min1 | sgn, min2) per check
//                           when it fits (read by successor checks for B2V)
//                workspace  Q*_v of weight-1 columns; (position, 64 sign bits) per check
//                           [, (min1 | sgn, min2) per check]
//   layered NMS: shared     Lambda_v of weight >= 2 columns
//                workspace  Lambda_v of weight-1 columns; (min1 | sgn, min2, position,
//                           32 sign bits) per check
#include "cbp_kernel_common.cuh"

namespace cbp {
namespace {

constexpr float kInf = __builtin_huge_valf();

// CBP min-sum: lane z's slots of base entry `se` (the CBP-SP kernel's records,
// lane-independent parts precomputed): its variable's state (weight >= 2 columns: position (z + s) mod Z of the
// column; weight 1: the check lane's own slot) and its predecessor check.
__device__ __forceinline__ int var_slot(const SpEdge& se, int z, int Z) {
  return static_cast<int>(se.x & kSpMask) + z - (z >= static_cast<int>(se.w & 0xffffu) ? Z : 0);
}
__device__ __forceinline__ int pred_off(const SpEdge& se, int z, int Z) {
  return z - (z >= static_cast<int>(se.w >> 16) ? Z : 0);
}

// Layered NMS on one check (lane z, check m = r*Z + z, d <= D edges): pass 1 forms
// Q = Lambda - R_old (Eq. s2e10) and the minima, pass 2 forms R_new and
// Lambda = Q + R_new (Eq. s2e12).  The V2C messages of the row stay in registers.
template <int D>
__device__ __forceinline__ void lbp_row(const BaseEdge* __restrict__ s_e, int k0, int d, int m,
                                        int z, int Z, int t, float alpha, float* VAR, float* SV,
                                        uint4* AUX) {
  float r1 = 0.0f, r2 = 0.0f;
  uint32_t osig = 0, oidx = 0, osg = 0;
  if (t > 1) {  // rebuild R_old from the check's state of the previous sweep
    const uint4 a = AUX[m];
    r1 = __fmul_rn(alpha, fabsf(__uint_as_float(a.x)));
    r2 = __fmul_rn(alpha, __uint_as_float(a.y));
    osig = a.x >> 31;
    oidx = a.z;
    osg = a.w;
  }
  float qv[D];
  float m1 = kInf, m2 = kInf;
  uint32_t idx = 0, sig = 0, sg = 0;
#pragma unroll
  for (int j = 0; j < D; ++j) {
    if (j < d) {
      const BaseEdge be = s_e[k0 + j];
      const int cidx = be.pad & 0xffff;
      const float lam = (be.flags & kSelf) ? SV[cidx * Z + z]
                                           : VAR[cidx * Z + mod_add(z + be.s, Z)];
      float rold = 0.0f;
      if (t > 1) {
        const float rm = (static_cast<uint32_t>(j) == oidx) ? r2 : r1;
        rold = (osig ^ ((osg >> j) & 1u)) ? -rm : rm;
      }
      const float q = __fsub_rn(lam, rold);
      qv[j] = q;
      const float a = fabsf(q);
      if (a < m1) {
        m2 = m1;
        m1 = a;
        idx = j;
      } else if (a < m2) {
        m2 = a;
      }
      const uint32_t neg = q < 0.0f;
      sig ^= neg;
      sg |= neg << j;
    }
  }
  const float n1 = __fmul_rn(alpha, m1), n2 = __fmul_rn(alpha, m2);
#pragma unroll
  for (int j = 0; j < D; ++j) {
    if (j < d) {
      const BaseEdge be = s_e[k0 + j];
      const int cidx = be.pad & 0xffff;
      const float rm = (static_cast<uint32_t>(j) == idx) ? n2 : n1;
      const float lam = __fadd_rn(qv[j], (sig ^ ((sg >> j) & 1u)) ? -rm : rm);
      if (be.flags & kSelf) SV[cidx * Z + z] = lam;
      else VAR[cidx * Z + mod_add(z + be.s, Z)] = lam;
    }
  }
  AUX[m] = make_uint4(__float_as_uint(sig ? -m1 : m1), __float_as_uint(m2), idx, sg);
}

// RST (CBP min-sum only): the C2V messages are kept per edge in the workspace, R [base
// entry][lane] as in the CBP log-tanh kernel: B2V stores R^new in the predecessor's slot
// (Eq. s4e22) and V2C reads the edge's own slot, so the check state shrinks to
// (min1 | sgn, min2) and no old message is rebuilt.
template <int ALG, bool CHKS, int MAXT, bool RST = false>
__global__ void __launch_bounds__(MAXT, 1) minsum_kernel(const KParams p) {
  constexpr bool CBP = (ALG == ALG_CBP_NMS);
  static_assert(!RST || CBP, "per-edge messages: CBP min-sum only");
  extern __shared__ __align__(16) unsigned char smem[];
  const int Z = p.Z, N = p.N, M = p.M, words = p.words, G = p.F;
  const int tid = threadIdx.x;
  const int g = tid / Z;
  const int z = tid - g * Z;
  const bool lane = g < G;
  const float alpha = p.alpha;

  unsigned char* sp = smem;
  BaseEdge* s_e = reinterpret_cast<BaseEdge*>(sp);
  sp += sizeof(BaseEdge) * p.nnzb;
  // CBP min-sum: the per-entry lane records of the CBP-SP kernel (two slots per edge: the
  // variable's and the predecessor check's; layered min-sum, with one, keeps the plain list)
  SpEdge* s_spe = reinterpret_cast<SpEdge*>(sp);
  if (CBP) sp += sizeof(SpEdge) * p.nnzb;
  int* s_rptr = reinterpret_cast<int*>(sp);
  sp += sizeof(int) * ((p.mb + 1 + 3) & ~3);
  uint2* s_col = reinterpret_cast<uint2*>(sp);  // (last row | shift << 16, idx | self << 16)
  sp += sizeof(uint2) * ((p.nb + 1) & ~1);
  SlotState* s_slot = reinterpret_cast<SlotState*>(sp);
  sp += sizeof(SlotState) * ((G + 3) & ~3);
  float* s_groups = reinterpret_cast<float*>(sp);

  for (int i = tid; i < p.nnzb; i += blockDim.x) {
    s_e[i] = p.edges[i];
    if (CBP) s_spe[i] = p.spe[i];
  }
  for (int i = tid; i <= p.mb; i += blockDim.x) s_rptr[i] = p.rptr[i];
  for (int c = tid; c < p.nb; c += blockDim.x) {
    const ColEntry ce = p.cols[p.cptr[c + 1] - 1];
    const BaseEdge be = p.edges[ce.e];
    s_col[c] = make_uint2(uint32_t(ce.r) | (uint32_t(ce.s) << 16),
                          (be.pad & 0xffffu) | ((be.flags & kSelf) ? 0x10000u : 0u));
  }
  for (int k = tid; k < G; k += blockDim.x) {
    s_slot[k].frame = blockIdx.x * G + k;
    s_slot[k].t = 0;
    s_slot[k].unsat = 0;
  }
  // per group, shared: VAR [ncomp*Z] | CHK [M] float2 (CBP, CHKS) | bits [wpad]
  float* gbase = s_groups + static_cast<size_t>(lane ? g : 0) * p.sh_frame;
  float* VAR = gbase;
  float* nxt = gbase + ((static_cast<size_t>(p.ncomp) * Z + 3) & ~static_cast<size_t>(3));
  const long long gslot = static_cast<long long>(blockIdx.x) * G + (lane ? g : 0);
  float* wsl = p.ws + gslot * p.ws_slot;
  float* SV = wsl + p.ws_off_sv;                          // [nself*Z]
  uint4* AUX = reinterpret_cast<uint4*>(wsl + p.ws_off_s);  // [M] (not RST)
  float* Rg = wsl + p.ws_off_s;                           // [E] (RST)
  float2* CHK = nullptr;                                  // [M] (CBP)
  if (CBP) {
    if (CHKS) {
      CHK = reinterpret_cast<float2*>(nxt);
      nxt += 2 * ((M + 1) & ~1);
    } else {
      CHK = reinterpret_cast<float2*>(wsl + p.ws_off_c);
    }
  }
  uint32_t* bits = reinterpret_cast<uint32_t*>(nxt);
  SlotState* my = s_slot + (lane ? g : 0);
  if (lane)
    for (int w = z; w < ((words + 3) & ~3); w += Z) bits[w] = 0u;
  const int tg = p.team_groups;
  const bool single_team = tg >= G;
  const int bar_id = single_team ? 0 : 1 + (lane ? g / tg : 0);
  const int bar_n = single_team ? static_cast<int>(blockDim.x) : tg * Z;
  __syncthreads();

  for (;;) {
    const int frame = lane ? my->frame : p.batch;
    const bool act = frame < p.batch;
    if (act && my->t == 0) {  // Q*_v = L_v (CBP, Eq. s4e15); Lambda_v = L_v (LBP)
      const float* src = p.llr + static_cast<long long>(frame) * N;
      bool bad = false;
      constexpr int LB = 4;  // the loads of a block of columns are issued together
      for (int c0 = 0; c0 < p.nb; c0 += LB) {
        float Lb[LB];
#pragma unroll
        for (int u = 0; u < LB; ++u) {
          const int c = c0 + u;
          if (c < p.nb) {
            const uint2 ci = s_col[c];
            Lb[u] = __ldg(src + c * Z +
                          ((ci.y & 0x10000u) ? mod_add(z + int(ci.x >> 16), Z) : z));
          }
        }
#pragma unroll
        for (int u = 0; u < LB; ++u) {
          const int c = c0 + u;
          if (c < p.nb) {
            const uint2 ci = s_col[c];
            const int idx = ci.y & 0xffff;
            const float L = Lb[u];
            bad |= non_finite(L);
            if (ci.y & 0x10000u) SV[idx * Z + z] = L;
            else VAR[idx * Z + z] = L;
          }
        }
      }
      if (bad) atomicOr(p.status, kStatusNonFiniteLlr);
    }
    if (!team_sync_or(bar_id, bar_n, act)) break;
    const int t = act ? my->t + 1 : 0;

    for (int r = 0; r < p.mb; ++r) {
      if (act) {
        if (!RST && t > 1 && z == 0) {
          // the check states of base row r + 1 (cyclically) are contiguous in the
          // workspace: one bulk L2 prefetch per lane group brings them on chip while this
          // row runs (a non-binding hint), and the state block of that row's weight-1
          // column when it ends the row
          const int rn = r + 1 < p.mb ? r + 1 : 0;
          const float* a = reinterpret_cast<const float*>(AUX + rn * Z);
          prefetch_l2(a, a + 4 * Z);
          const BaseEdge bl = s_e[s_rptr[rn + 1] - 1];
          if (bl.flags & kSelf) {
            const float* sv = SV + (bl.pad & 0xffff) * Z;
            prefetch_l2(sv, sv + Z);
          }
        }
        const int k0 = s_rptr[r], d = s_rptr[r + 1] - k0;
        const int m = r * Z + z;
        if (CBP) {
          // own state from the previous sweep: rebuilds R_{c_i->v} (Eq. s4e19)
          float r1 = 0.0f, r2 = 0.0f;
          uint32_t osig = 0, oidx = 0;
          unsigned long long osg = 0;
          if (!RST && t > 1) {
            const float2 cs = CHK[m];
            const uint4 a = AUX[m];
            r1 = __fmul_rn(alpha, fabsf(cs.x));
            r2 = __fmul_rn(alpha, cs.y);
            osig = sign_bit(cs.x);
            oidx = a.x;
            osg = (static_cast<unsigned long long>(a.z) << 32) | a.y;
          }
          float m1 = kInf, m2 = kInf;
          uint32_t idx = 0, sig = 0;
          unsigned long long sg = 0;
          for (int j0 = 0; j0 < d; j0 += 4) {
            float q[4], ro[4];
            float2 pc[4];
            int qoff[4], roff[4];
            uint32_t fl[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) {
              const int j = j0 + u;
              if (j < d) {
                const SpEdge se = s_spe[k0 + j];
                const int pz = pred_off(se, z, Z);
                fl[u] = se.x;
                qoff[u] = var_slot(se, z, Z);
                q[u] = (se.x & kSpSelf) ? SV[qoff[u]] : VAR[qoff[u]];
                pc[u] = CHK[static_cast<int>(se.y) + pz];
                if (RST) {  // own slot (c_i -> v), predecessor slot (c_j -> v)
                  ro[u] = (t > 1 && !(se.x & kSpSelf)) ? Rg[(k0 + j) * Z + z] : 0.0f;
                  roff[u] = static_cast<int>(se.z) + pz;
                }
              }
            }
#pragma unroll
            for (int u = 0; u < 4; ++u) {
              const int j = j0 + u;
              if (j < d) {
                // B2V, Eq. (s4e18xx): min2 of c_j when |Q*_v| is its min1
                float Rn = 0.0f;
                if (!(t == 1 && (fl[u] & kSpFirst))) {
                  const float b1 = fabsf(pc[u].x);
                  const float rm = __fmul_rn(alpha, (fabsf(q[u]) == b1) ? pc[u].y : b1);
                  Rn = (sign_bit(pc[u].x) ^ (q[u] < 0.0f)) ? -rm : rm;
                }
                float rold = 0.0f;
                if (fl[u] & kSpSelf) {
                  rold = Rn;                                   // c_j == c_i
                } else if (RST) {
                  rold = ro[u];
                  if (!(t == 1 && (fl[u] & kSpFirst))) Rg[roff[u]] = Rn;  // Eq. (s4e22)
                } else if (t > 1) {
                  const float rm = (static_cast<uint32_t>(j) == oidx) ? r2 : r1;
                  rold = (osig ^ static_cast<uint32_t>((osg >> j) & 1ull)) ? -rm : rm;
                }
                const float qn = __fsub_rn(__fadd_rn(q[u], Rn), rold);  // Eq. (s4e19)
                const float a = fabsf(qn);                              // C2B, Eq. (s4e21xx)
                if (a < m1) {
                  m2 = m1;
                  m1 = a;
                  idx = j;
                } else if (a < m2) {
                  m2 = a;
                }
                const uint32_t neg = qn < 0.0f;
                sig ^= neg;
                if (!RST) sg |= static_cast<unsigned long long>(neg) << j;
                if (fl[u] & kSpSelf) SV[qoff[u]] = qn;
                else VAR[qoff[u]] = qn;
              }
            }
          }
          CHK[m] = make_float2(sig ? -m1 : m1, m2);
          if (!RST)
            AUX[m] = make_uint4(idx, static_cast<uint32_t>(sg), static_cast<uint32_t>(sg >> 32), 0u);
        } else {
          // layered NMS, unrolled for the smallest degree bucket that holds the row
          if (d <= 8) lbp_row<8>(s_e, k0, d, m, z, Z, t, alpha, VAR, SV, AUX);
          else if (d <= 16) lbp_row<16>(s_e, k0, d, m, z, Z, t, alpha, VAR, SV, AUX);
          else lbp_row<kMaxDeg>(s_e, k0, d, m, z, Z, t, alpha, VAR, SV, AUX);
        }
      }
      team_sync(bar_id, bar_n);
    }

    // ---- posterior and hard decisions (Eq. s2e7), syndrome stop.  As in the CBP
    // log-tanh kernel, the checks of one base row (the test row) are evaluated first;
    // when one fails, the frame goes on without the full flush and syndrome scan.
    if (lane && z == 0) my->unsat = 0;
    team_sync(bar_id, bar_n);
    if (act && p.stop == CBP_STOP_SYNDROME && t < p.max_iter) {
      uint32_t par = 0;
      const int tk0 = s_rptr[p.test_row], tk1 = s_rptr[p.test_row + 1];
#pragma unroll 1
      for (int k = tk0; k < tk1; ++k) {
        const BaseEdge be = s_e[k];
        const uint2 ci = s_col[be.c];
        const int cidx = ci.y & 0xffff;
        const int sk = int(ci.x >> 16), rk = int(ci.x & 0xffff);
        float q;
        int ck;
        if (ci.y & 0x10000u) {
          q = SV[cidx * Z + z];
          ck = rk * Z + z;
        } else {
          const int a = mod_add(z + be.s, Z);
          q = VAR[cidx * Z + a];
          int zk = a - sk;
          zk = zk < 0 ? zk + Z : zk;
          ck = rk * Z + zk;
        }
        float lb = q;
        if (CBP) {
          const float2 pc = CHK[ck];
          const float b1 = fabsf(pc.x);
          const float rm = __fmul_rn(alpha, (fabsf(q) == b1) ? pc.y : b1);
          lb = __fadd_rn(q, (sign_bit(pc.x) ^ (q < 0.0f)) ? -rm : rm);
        }
        par ^= lb < 0.0f ? 1u : 0u;
      }
      if (par) my->unsat = 1;
    }
    team_sync(bar_id, bar_n);
    const bool full =
        act && (t >= p.max_iter || (p.stop == CBP_STOP_SYNDROME &&
                                    *static_cast<volatile int*>(&my->unsat) == 0));
    // a frame tested in full most likely stops now: ask L2 for the channel LLRs of its
    // slot's next frame while the flush and the syndrome scan run
    if (full && z == 0 && frame + p.slots < p.batch) {
      const float* nx = p.llr + static_cast<long long>(frame + p.slots) * N;
      for (int o = 0; o < N; o += 8192) prefetch_l2(nx + o, nx + min(o + 8192, N));
    }
    // the decision bits are zero here (cleared at the start and after each full test);
    // the warp skips the flush when none of its frames needs it
    if (__any_sync(0xffffffffu, full)) {
      constexpr int FC = 2;  // columns per block: the block's loads are issued together
      for (int c0 = 0; c0 < p.nb; c0 += FC) {
        float qb[FC];
        float2 pcb[FC];
        int vb[FC];
#pragma unroll
        for (int u = 0; u < FC; ++u) {
          const int c = c0 + u;
          vb[u] = 0;
          if (full && c < p.nb) {
            const uint2 ci = s_col[c];
            const int cidx = ci.y & 0xffff;
            const int sk = int(ci.x >> 16), rk = int(ci.x & 0xffff);
            int ck;
            if (ci.y & 0x10000u) {  // weight-1 column: lane z owns its single check (rk, z)
              qb[u] = SV[cidx * Z + z];
              ck = rk * Z + z;
              vb[u] = c * Z + mod_add(z + sk, Z);
            } else {
              qb[u] = VAR[cidx * Z + z];
              int zk = z - sk;
              zk = zk < 0 ? zk + Z : zk;
              ck = rk * Z + zk;
              vb[u] = c * Z + z;
            }
            if (CBP) pcb[u] = CHK[ck];
          }
        }
#pragma unroll
        for (int u = 0; u < FC; ++u) {
          if (c0 + u >= p.nb) break;  // uniform across the warp
          const int v = vb[u];
          bool neg = false;
          if (full) {
            const float q = qb[u];
            float lb = q;
            if (CBP) {  // flushed posterior: Eq. (s4e20) with the last check of v as c_j
              const float2 pc = pcb[u];
              const float b1 = fabsf(pc.x);
              const float rm = __fmul_rn(alpha, (fabsf(q) == b1) ? pc.y : b1);
              lb = __fadd_rn(q, (sign_bit(pc.x) ^ (q < 0.0f)) ? -rm : rm);
            }
            neg = lb < 0.0f;
            if (p.soft) p.soft[static_cast<long long>(frame) * N + v] = lb;
          }
          warp_or_bit(bits + (v >> 5), neg ? (1u << (v & 31)) : 0u, full);
        }
      }
    }
    team_sync(bar_id, bar_n);
    // ---- syndrome; a frame stops scanning at its first unsatisfied check row
    if (full) {
      for (int r = 0; r < p.mb; ++r) {
        uint32_t pr = 0;
        for (int k = s_rptr[r]; k < s_rptr[r + 1]; ++k) {
          const BaseEdge be = s_e[k];
          const int v = be.c * Z + mod_add(z + be.s, Z);
          pr ^= bits[v >> 5] >> (v & 31);
        }
        if (pr & 1u) my->unsat = 1;
        if (*static_cast<volatile int*>(&my->unsat)) break;
      }
    }
    team_sync(bar_id, bar_n);
    bool done = false;
    if (full) {
      const bool ok = my->unsat == 0;
      done = (ok && p.stop == CBP_STOP_SYNDROME) || t >= p.max_iter;
      if (done) {
        uint32_t* ho = p.hard + static_cast<long long>(frame) * words;
        for (int w = z; w < words; w += Z) ho[w] = bits[w];
        if (z == 0) p.iters[frame] = ok ? t : -t;
      }
    }
    team_sync(bar_id, bar_n);
    if (full)  // ready for the next full test
      for (int w = z; w < words; w += Z) bits[w] = 0u;
    if (act && z == 0) {
      if (done) {
        my->frame = frame + p.slots;
        my->t = 0;
      } else {
        my->t = t;
      }
    }
    team_sync(bar_id, bar_n);
  }
}

}  // namespace

void* minsum_kernel_ptr(int alg, bool chk_shared, bool rstore) {
  if (alg == ALG_CBP_NMS && rstore)
    return chk_shared ? reinterpret_cast<void*>(&minsum_kernel<ALG_CBP_NMS, true, 768, true>)
                      : reinterpret_cast<void*>(&minsum_kernel<ALG_CBP_NMS, false, 768, true>);
  if (alg == ALG_CBP_NMS)
    return chk_shared ? reinterpret_cast<void*>(&minsum_kernel<ALG_CBP_NMS, true, 768>)
                      : reinterpret_cast<void*>(&minsum_kernel<ALG_CBP_NMS, false, 768>);
  return reinterpret_cast<void*>(&minsum_kernel<ALG_LBP_NMS, false, 768>);
}

}  // namespace cbp
