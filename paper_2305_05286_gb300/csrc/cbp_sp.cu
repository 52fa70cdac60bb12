// CBP, log-tanh form (Sec. IV-C, Steps 1-3): the main decoder kernel on sm_103a.
//
// A CTA holds G lane groups of Z lanes; lane z of a group owns check r*Z + z of every
// base row r for FPT frames at once (FPT = 1 or 2).  The Z checks of a base row share
// no variable, so they run in parallel and one barrier per base row keeps the paper's
// sequential order exactly.  The FPT frames of a group are independent: each has its
// own sweep counter, stops on its own syndrome and is replaced by the next frame of its
// slot at the following sweep boundary; they only share the index arithmetic and the
// memory instructions, because their state is interleaved frame-innermost:
//   shared    (Q*_v, phi(|Q*_v|)) per frame for the variables of weight >= 2 columns,
//             [compact column][lane][frame]; the check-beliefs S_c (sign bit = sgn
//             Omega_c) [check][frame] when they fit; decision bits per frame
//   workspace C2V messages R [base entry][lane][frame]; (Q*, phi) of weight-1 columns,
//             which only their one check lane touches, [column][lane][frame]; S_c when
//             not shared
// A base row is processed in chunks of CH edges: the loads of a chunk are issued
// together, then the CH edge updates run with independent phi evaluations, in
// ascending column order (the order of the C2B fold).  While a row runs, one thread per
// group asks L2 for the next row's C2V block and weight-1 state block (bulk prefetches,
// no data dependence).
//
// Kernels of this file, all on the same sweep body (sp_body):
//   cbp_sp_kernel        one code, frames spread over persistent frame slots
//   cbp_sp_win_kernel    the same with the paper's own stop, Eq. (s4e24), and the
//                        Step 3 output (one frame per group, extra barriers per row)
//   cbp_sp_multi_kernel  several codes in one launch: CTAs take (code, frame range)
//                        chunks from a work counter
#include "cbp_kernel_common.cuh"

namespace cbp {
namespace {

// Vector access to FPT interleaved frames.
template <int FPT> struct Lanes;
template <> struct Lanes<1> {
  __device__ static void ld_pair(const float* a, int i, float* q, float* p) {
    const float2 v = reinterpret_cast<const float2*>(a)[i];
    q[0] = v.x; p[0] = v.y;
  }
  __device__ static void st_pair(float* a, int i, const float* q, const float* p) {
    reinterpret_cast<float2*>(a)[i] = make_float2(q[0], p[0]);
  }
  __device__ static void ld(const float* a, int i, float* x) { x[0] = a[i]; }
  __device__ static void st(float* a, int i, const float* x) { a[i] = x[0]; }
};
template <> struct Lanes<2> {
  __device__ static void ld_pair(const float* a, int i, float* q, float* p) {
    const float4 v = reinterpret_cast<const float4*>(a)[i];
    q[0] = v.x; p[0] = v.y; q[1] = v.z; p[1] = v.w;
  }
  __device__ static void st_pair(float* a, int i, const float* q, const float* p) {
    reinterpret_cast<float4*>(a)[i] = make_float4(q[0], p[0], q[1], p[1]);
  }
  __device__ static void ld(const float* a, int i, float* x) {
    const float2 v = reinterpret_cast<const float2*>(a)[i];
    x[0] = v.x; x[1] = v.y;
  }
  __device__ static void st(float* a, int i, const float* x) {
    reinterpret_cast<float2*>(a)[i] = make_float2(x[0], x[1]);
  }
};

// Registers of one chunk of CH edges of a base row (FPT frames each).
template <int FPT, int CH>
struct Chunk {
  float q[CH][FPT], ph[CH][FPT], sj[CH][FPT], ro[CH][FPT];
  int qoff[CH];   // pair index of the variable in QP (weight >= 2) or SV (weight 1)
  int roff[CH];   // predecessor R slot (base entry of c_j, lane of c_j)
  uint32_t fl[CH];
  int vidx[CH];   // variable index (paper-literal stop only)
};

// Loads of a chunk: (Q*, phi) of each variable, S of its predecessor check c_j, and
// the edge's own R slot (read only once the frame is past its first sweep).
template <int FPT, int CH, bool WIN, bool NOSELF = false>
__device__ __forceinline__ void load_chunk(Chunk<FPT, CH>& c, int kb, int k1,
                                           const SpEdge* __restrict__ s_spe, int z, int Z,
                                           bool later, const float* QP, const float* SV,
                                           const float* S, const float* R,
                                           const BaseEdge* __restrict__ g_edges) {
  using LV = Lanes<FPT>;
#pragma unroll
  for (int j = 0; j < CH; ++j) {
    const int k = kb + j;
    if (k < k1) {
      const SpEdge se = s_spe[k];
      const int tq = static_cast<int>(se.w & 0xffffu), tj = static_cast<int>(se.w >> 16);
      const int uj = z >= tj ? Z : 0;
      c.fl[j] = se.x;
      c.qoff[j] = static_cast<int>(se.x & kSpMask) + z - (z >= tq ? Z : 0);
      c.roff[j] = static_cast<int>(se.z) + z - uj;
      if (!NOSELF && (se.x & kSpSelf)) {
        LV::ld_pair(SV, c.qoff[j], c.q[j], c.ph[j]);
      } else {
        LV::ld_pair(QP, c.qoff[j], c.q[j], c.ph[j]);
        if (later) LV::ld(R, k * Z + z, c.ro[j]);
      }
      LV::ld(S, static_cast<int>(se.y) + z - uj, c.sj[j]);
      if (WIN) {
        const BaseEdge be = g_edges[k];
        c.vidx[j] = be.c * Z + mod_add(z + be.s, Z);
      }
    }
  }
}

// Step 2 (1) b)-e) for the edges of a chunk, in ascending column order.  Signs are
// handled on the sign bits: no Q* is ever -0 (the channel LLRs are loaded as L + 0,
// and a sum or difference of values that are not -0 is -0 only when both are -0 and
// R^new is never -0), so the sign bit of Q* is [Q* < 0].
// WIN (paper-literal stop, one frame per group): the posterior Lambda = Q* + R^new of
// Eq. (s4e20) is compared with the variable's previous one (sign bit in pbits); a flip
// toggles the bit and is recorded in fmask (bit = edge position in the row).
template <int FPT, int CH, bool WIN, bool NOSELF = false>
__device__ __forceinline__ void update_chunk(const Chunk<FPT, CH>& c, int kb, int k1,
                                             const int* t, float* Sacc, uint32_t* sig,
                                             float xlo, const float4* __restrict__ tab,
                                             float* QP, float* SV, float* R, uint32_t* pbits,
                                             int k0, uint32_t& fmask) {
  using LV = Lanes<FPT>;
#pragma unroll
  for (int j = 0; j < CH; ++j) {
    if (kb + j < k1) {
      const bool self = !NOSELF && (c.fl[j] & kSpSelf);
      const bool first_row = c.fl[j] & kSpFirst;
      float Rn[FPT], qn[FPT], phn[FPT];
      bool store_r = false;
#pragma unroll
      for (int h = 0; h < FPT; ++h) {
        // B2V, Eqs. (s4e18), (s4e13): exclude phi(|Q*|) from S of c_j; a variable not
        // visited before adds no C2V
        const float mag = phi_eval(fabsf(__fsub_rn(fabsf(c.sj[j][h]), c.ph[j][h])), xlo, tab);
        const float rb = __uint_as_float(__float_as_uint(mag) |
                                         ((__float_as_uint(c.sj[j][h]) ^
                                           __float_as_uint(c.q[j][h])) & 0x80000000u));
        const bool first = (t[h] == 1) && first_row;
        Rn[h] = first ? 0.0f : rb;
        store_r |= !first;
        // V2C, Eqs. (s4e20), (s4e19); weight-1 column: c_j == c_i
        const float rold = self ? Rn[h] : (t[h] > 1 ? c.ro[j][h] : 0.0f);
        const float lam = __fadd_rn(c.q[j][h], Rn[h]);
        qn[h] = __fsub_rn(lam, rold);
        if (WIN) {  // Eq. (s4e24): did the posterior's sign flip?
          const int v = c.vidx[j];
          const uint32_t bit = 1u << (v & 31);
          const bool neg = __float_as_uint(lam) >> 31;
          if (neg != ((pbits[v >> 5] & bit) != 0)) {
            atomicXor(pbits + (v >> 5), bit);
            fmask |= 1u << (kb + j - k0);
          }
        }
        // C2B, Eq. (s4e21) as a sum of phi; the sign bits fold into sig
        phn[h] = phi_eval(fabsf(qn[h]), xlo, tab);
        Sacc[h] = __fadd_rn(Sacc[h], phn[h]);
        sig[h] ^= __float_as_uint(qn[h]);
      }
      if (self) {
        LV::st_pair(SV, c.qoff[j], qn, phn);
      } else {
        if (store_r) LV::st(R, c.roff[j], Rn);  // R_{c_j->v} <- R^new (Eq. s4e22)
        LV::st_pair(QP, c.qoff[j], qn, phn);
      }
    }
  }
}

// One base row of CH-edge chunks: loads of the next chunk are issued before the
// current chunk's updates when DB (they never alias: a row reads its own R slots, the
// beliefs of other rows and distinct variables, and writes predecessor R slots, its
// variables and its own beliefs).
// SELFLAST: the code's weight-1 edges are each the last edge of their row (one per row at
// most, checked on the host), so the chunk loop runs without the weight-1 branches and
// that edge follows on its own -- still last in the column order of the fold.
template <int FPT, int CH, bool DB, bool WIN, bool SELFLAST>
__device__ __forceinline__ void row_edges(int k0, int k1, const SpEdge* __restrict__ s_spe,
                                          int z, int Z, bool later, const int* t, float* Sacc,
                                          uint32_t* sig, float xlo,
                                          const float4* __restrict__ tab, float* QP, float* SV,
                                          const float* S, float* R,
                                          const BaseEdge* __restrict__ g_edges, uint32_t* pbits,
                                          uint32_t& fmask) {
  if (DB) {
    Chunk<FPT, CH> A, B;
    load_chunk<FPT, CH, WIN>(A, k0, k1, s_spe, z, Z, later, QP, SV, S, R, g_edges);
    for (int kb = k0;;) {
      if (kb + CH < k1)
        load_chunk<FPT, CH, WIN>(B, kb + CH, k1, s_spe, z, Z, later, QP, SV, S, R, g_edges);
      update_chunk<FPT, CH, WIN>(A, kb, k1, t, Sacc, sig, xlo, tab, QP, SV, R, pbits, k0,
                                 fmask);
      kb += CH;
      if (kb >= k1) break;
      if (kb + CH < k1)
        load_chunk<FPT, CH, WIN>(A, kb + CH, k1, s_spe, z, Z, later, QP, SV, S, R, g_edges);
      update_chunk<FPT, CH, WIN>(B, kb, k1, t, Sacc, sig, xlo, tab, QP, SV, R, pbits, k0,
                                 fmask);
      kb += CH;
      if (kb >= k1) break;
    }
  } else if (SELFLAST) {
    const bool has_self = (s_spe[k1 - 1].x & kSpSelf) != 0;
    const int km = has_self ? k1 - 1 : k1;
    int kb = k0;
    for (; kb + CH <= km; kb += CH) {  // whole chunks: the edge guards fold away
      Chunk<FPT, CH> A;
      load_chunk<FPT, CH, WIN, true>(A, kb, kb + CH, s_spe, z, Z, later, QP, SV, S, R,
                                     g_edges);
      update_chunk<FPT, CH, WIN, true>(A, kb, kb + CH, t, Sacc, sig, xlo, tab, QP, SV, R,
                                       pbits, k0, fmask);
    }
    if (kb < km) {  // the remainder, guarded
      Chunk<FPT, CH> A;
      load_chunk<FPT, CH, WIN, true>(A, kb, km, s_spe, z, Z, later, QP, SV, S, R, g_edges);
      update_chunk<FPT, CH, WIN, true>(A, kb, km, t, Sacc, sig, xlo, tab, QP, SV, R, pbits, k0,
                                       fmask);
    }
    if (has_self) {
      Chunk<FPT, 1> A;
      load_chunk<FPT, 1, WIN>(A, k1 - 1, k1, s_spe, z, Z, later, QP, SV, S, R, g_edges);
      update_chunk<FPT, 1, WIN>(A, k1 - 1, k1, t, Sacc, sig, xlo, tab, QP, SV, R, pbits, k0,
                                fmask);
    }
  } else {
    for (int kb = k0; kb < k1; kb += CH) {
      Chunk<FPT, CH> A;
      load_chunk<FPT, CH, WIN>(A, kb, k1, s_spe, z, Z, later, QP, SV, S, R, g_edges);
      update_chunk<FPT, CH, WIN>(A, kb, k1, t, Sacc, sig, xlo, tab, QP, SV, R, pbits, k0,
                                 fmask);
    }
  }
}

constexpr int kPrefetchRows = 1;

// Paper-literal stop: one thread of a lane group walks the row's check updates in order
// (lane z = check r*Z + z) with the window counter wst[0]; wst[1] receives the lane at
// which the counter reaches M, or -1.  ok[z] = 1 if check z left Omega > 0 and flipped
// no posterior sign.
__device__ __forceinline__ void window_scan(const unsigned char* ok, int Z, int M, int* wst) {
  int run = wst[0], stop = -1, i = 0;
  for (; i + 4 <= Z && stop < 0; i += 4) {
    if (*reinterpret_cast<const uint32_t*>(ok + i) == 0x01010101u) {
      if (run + 4 >= M) stop = i + (M - run - 1);
      else run += 4;
    } else {
      for (int b = 0; b < 4 && stop < 0; ++b)
        if (!ok[i + b]) run = 0;
        else if (++run >= M) stop = i + b;
    }
  }
  for (; i < Z && stop < 0; ++i)
    if (!ok[i]) run = 0;
    else if (++run >= M) stop = i;
  wst[0] = stop < 0 ? run : M;
  wst[1] = stop;
}

// Step 2 of one sweep: the base rows in order, one team barrier after each.  WIN adds
// the window test of Eq. (s4e24) after every row (two more team barriers, executed by
// every thread of the team); a group whose window fills stops in the middle of the row
// at that check: lanes after it undo their posterior-sign updates, and `halted` keeps
// the group idle for the rest of the sweep.
template <int FPT, int CH, bool DB, bool WIN, bool SELFLAST>
__device__ __forceinline__ void sweep_rows(int mb, bool any, const int* s_rptr,
                                           const SpEdge* __restrict__ s_spe, int z, int Z,
                                           bool later, const int* t, float xlo,
                                           const float4* __restrict__ tab, float* QP, float* SV,
                                           float* S, float* R, int bar_id, int bar_n,
                                           const BaseEdge* __restrict__ g_edges,
                                           uint32_t* pbits, int* wst, unsigned char* okb, int M,
                                           bool& halted) {
  using LV = Lanes<FPT>;
  for (int r = 0; r < mb; ++r) {
    const bool work = any && !(WIN && halted);
    const int k0 = s_rptr[r], k1 = s_rptr[r + 1];
    uint32_t fmask = 0, sig0 = 0;
    if (work) {
      if (later && z == 0) {
        // the C2V slots of base row r + kPrefetchRows (cyclically) are contiguous in the
        // workspace: one bulk L2 prefetch per lane group brings them on chip while this
        // row runs (a non-binding hint; rows in between may still rewrite those lines);
        // likewise the (Q*, phi) block of that row's weight-1 column
        int rn = r + kPrefetchRows;
        rn = rn >= mb ? rn - mb : rn;
        const float* a = R + static_cast<long long>(s_rptr[rn]) * Z * FPT;
        const float* b = R + static_cast<long long>(s_rptr[rn + 1]) * Z * FPT;
        prefetch_l2(a, b);
        if (FPT == 1) {  // and the state block of that row's weight-1 column, if any
          const uint32_t x = s_spe[s_rptr[rn + 1] - 1].x;
          if (x & kSpSelf) {
            const float* sv = SV + 2 * static_cast<long long>(x & kSpMask);
            prefetch_l2(sv, sv + 2 * Z);
          }
        }
      }
      float Sacc[FPT];
      uint32_t sig[FPT];
#pragma unroll
      for (int h = 0; h < FPT; ++h) {
        Sacc[h] = 0.0f;
        sig[h] = 0;
      }
      row_edges<FPT, CH, DB, WIN, SELFLAST>(k0, k1, s_spe, z, Z, later, t, Sacc, sig, xlo, tab,
                                            QP, SV, S, R, g_edges, pbits, fmask);
      float sv[FPT];
#pragma unroll
      for (int h = 0; h < FPT; ++h)  // Sacc >= 0: its sign bit is free for sgn(Omega)
        sv[h] = __uint_as_float(__float_as_uint(Sacc[h]) | (sig[h] & 0x80000000u));
      LV::st(S, r * Z + z, sv);  // Eq. (s4e23); the sign bit carries sgn(Omega)
      sig0 = sig[0];
    }
    if (WIN) {
      if (work) okb[z] = ((sig0 & 0x80000000u) == 0 && fmask == 0) ? 1 : 0;  // Eq. (s4e2)
      team_sync(bar_id, bar_n);
      if (work && z == 0) window_scan(okb, Z, M, wst);
      team_sync(bar_id, bar_n);
      if (work && wst[1] >= 0) {
        if (z > wst[1])  // checks after the stop point were not yet updated
          for (int k = k0; k < k1; ++k)
            if ((fmask >> (k - k0)) & 1u) {
              const BaseEdge be = g_edges[k];
              const int v = be.c * Z + mod_add(z + be.s, Z);
              atomicXor(pbits + (v >> 5), 1u << (v & 31));
            }
        halted = true;
      }
    }
    team_sync(bar_id, bar_n);
  }
}

// Sweep-end pre-test: lane z evaluates the flushed posterior (Eq. s4e20, read-only) of
// each variable of check (test row, z) and folds its hard decision (Eq. s2e7) into
// par[h]; an odd par[h] is an unsatisfied check, so frame h's syndrome is non-zero.
// The variable of entry (r, c, s) is position a = (z + s) mod Z of column c; its last
// check is (rk, (a - sk) mod Z) for the last entry (rk, c, sk) of the column (for a
// weight-1 column: (r, z) itself, its state kept by lane z).
template <int FPT>
__device__ __forceinline__ void test_row_parity(const KParams& p, const int* s_rptr,
                                                const uint2* s_col, int z, int Z, float xlo,
                                                const float4* __restrict__ tab, const float* QP,
                                                const float* SV, const float* S, uint32_t* par) {
  using LV = Lanes<FPT>;
  const int k0 = s_rptr[p.test_row], k1 = s_rptr[p.test_row + 1];
#pragma unroll 1
  for (int k = k0; k < k1; ++k) {
    const BaseEdge be = p.edges[k];  // read through L1, like the syndrome scan
    const uint2 ci = s_col[be.c];
    const int idx = ci.y & 0xffff;
    const int sk = int(ci.x >> 16), rk = int(ci.x & 0xffff);
    float qv[FPT], pv[FPT], Sk[FPT];
    if (ci.y & 0x10000u) {
      LV::ld_pair(SV, idx * Z + z, qv, pv);
      LV::ld(S, rk * Z + z, Sk);
    } else {
      const int a = mod_add(z + be.s, Z);
      LV::ld_pair(QP, idx * Z + a, qv, pv);
      int zk = a - sk;
      zk = zk < 0 ? zk + Z : zk;
      LV::ld(S, rk * Z + zk, Sk);
    }
#pragma unroll
    for (int h = 0; h < FPT; ++h) {
      const float mag = phi_eval(fabsf(__fsub_rn(fabsf(Sk[h]), pv[h])), xlo, tab);
      const float lb = __fadd_rn(
          qv[h], __uint_as_float(__float_as_uint(mag) |
                                 ((__float_as_uint(Sk[h]) ^ __float_as_uint(qv[h])) &
                                  0x80000000u)));
      par[h] ^= lb < 0.0f ? 1u : 0u;
    }
  }
}

// Decode frames frame0, frame0 + 1, ... of one code with the lane groups of this CTA:
// frame slot k starts at frame0 + k and advances by `stride` when its frame stops, until
// it passes `end`.  Returns when every slot of the CTA is idle.
template <bool CHKS, int FPT, int CH, bool DB, bool WIN = false, bool SELFLAST = false>
__device__ __forceinline__ void sp_body(const KParams& p, int frame0, int stride, int end,
                                        unsigned char* smem, bool load_tab) {
  static_assert(!WIN || FPT == 1, "the paper-literal stop runs one frame per lane group");
  using LV = Lanes<FPT>;
  const int Z = p.Z, N = p.N, M = p.M, words = p.words, G = p.F;
  const int tid = threadIdx.x;
  const int g = tid / Z;
  const int z = tid - g * Z;
  const bool lane = g < G;

  unsigned char* sp = smem;
  float4* s_tab = reinterpret_cast<float4*>(sp);
  sp += sizeof(float4) * kPhiSegments;
  SpEdge* s_spe = reinterpret_cast<SpEdge*>(sp);
  sp += sizeof(SpEdge) * p.nnzb;
  int* s_rptr = reinterpret_cast<int*>(sp);
  sp += sizeof(int) * ((p.mb + 1 + 3) & ~3);
  uint2* s_col = reinterpret_cast<uint2*>(sp);  // (last row | shift << 16, idx | self << 16)
  sp += sizeof(uint2) * ((p.nb + 1) & ~1);
  SlotState* s_slot = reinterpret_cast<SlotState*>(sp);
  sp += sizeof(SlotState) * ((G * FPT + 3) & ~3);
  float* s_groups = reinterpret_cast<float*>(sp);

  if (load_tab)
    for (int i = tid; i < kPhiSegments; i += blockDim.x) s_tab[i] = p.phi_tab[i];
  for (int i = tid; i < p.nnzb; i += blockDim.x) s_spe[i] = p.spe[i];
  for (int i = tid; i <= p.mb; i += blockDim.x) s_rptr[i] = p.rptr[i];
  for (int c = tid; c < p.nb; c += blockDim.x) {
    const ColEntry ce = p.cols[p.cptr[c + 1] - 1];
    const BaseEdge be = p.edges[ce.e];
    s_col[c] = make_uint2(uint32_t(ce.r) | (uint32_t(ce.s) << 16),
                          (be.pad & 0xffffu) | ((be.flags & kSelf) ? 0x10000u : 0u));
  }
  for (int k = tid; k < G * FPT; k += blockDim.x) {
    s_slot[k].frame = frame0 + k;
    s_slot[k].t = 0;
    s_slot[k].unsat = 0;
  }
  // per group, shared: QP [ncomp*Z][FPT](Q,phi) | S [M][FPT] (CHKS) | bits [FPT][wpad]
  float* gbase = s_groups + static_cast<size_t>(lane ? g : 0) * p.sh_frame;
  float* QP = gbase;
  float* nxt = gbase + 2 * FPT * static_cast<size_t>(p.ncomp) * Z;
  // this CTA's workspace region, then the lane group's part of it
  float* wsl = p.ws + static_cast<long long>(blockIdx.x) * p.ws_cta +
               static_cast<long long>(lane ? g : 0) * p.ws_slot;
  float* R = wsl;                       // [E][FPT]
  float* SV = wsl + p.ws_off_sv;        // [nself*Z][FPT](Q,phi)
  float* S;
  if (CHKS) {
    S = nxt;
    nxt += FPT * ((M + 3) & ~3);
  } else {
    S = wsl + p.ws_off_s;
  }
  uint32_t* bits = reinterpret_cast<uint32_t*>(nxt);   // frame h: bits + h * wpad
  const int wpad = (words + 3) & ~3;
  // WIN: bits hold [latest posterior < 0] per variable; then the window counter and stop
  // lane (4 ints) and one ok byte per check lane
  int* wst = reinterpret_cast<int*>(bits + FPT * wpad);
  unsigned char* okb = reinterpret_cast<unsigned char*>(wst + 4);
  if (lane)  // WIN: [latest posterior < 0]; otherwise the decision bits of a full test
    for (int w = z; w < FPT * wpad; w += Z) bits[w] = 0u;
  SlotState* my = s_slot + (lane ? g : 0) * FPT;
  const float4* tab = s_tab;
  const float xlo = p.phi_xlo;
  const bool words_aligned = (Z & 31) == 0;
  // teams of p.team_groups lane groups (whole warps) synchronise among themselves
  const int tg = p.team_groups;
  const bool single_team = tg >= G || G * Z != static_cast<int>(blockDim.x);
  const int bar_id = single_team ? 0 : 1 + (lane ? g / tg : 0);
  const int bar_n = single_team ? static_cast<int>(blockDim.x) : tg * Z;
  __syncthreads();

  for (;;) {
    int frame[FPT], t[FPT];
    bool act[FPT];
    bool any = false;
#pragma unroll
    for (int h = 0; h < FPT; ++h) {
      frame[h] = lane ? my[h].frame : end;
      act[h] = frame[h] < end;
      any |= act[h];
      if (act[h] && my[h].t == 0) {  // Step 1, Eq. (s4e15): Q*_v = L_v for frame h
        const float* src = p.llr + static_cast<long long>(frame[h]) * N;
        bool bad = false;
        for (int c = 0; c < p.nb; ++c) {
          const uint2 ci = s_col[c];
          const int idx = ci.y & 0xffff;
          const int v =
              (ci.y & 0x10000u) ? c * Z + mod_add(z + int(ci.x >> 16), Z) : c * Z + z;
          const float L = __fadd_rn(__ldg(src + v), 0.0f);  // -0 -> +0
          bad |= non_finite(L);
          if (ci.y & 0x10000u)
            SV[((idx * Z + z) * FPT + h) * 2] = L;
          else
            QP[((idx * Z + z) * FPT + h) * 2] = L;
          if (WIN && L < 0.0f) atomicOr(bits + (v >> 5), 1u << (v & 31));
        }
        if (WIN && z == 0) wst[0] = 0;
        if (bad) atomicOr(p.status, kStatusNonFiniteLlr);
      }
    }
    if (!team_sync_or(bar_id, bar_n, any)) break;
#pragma unroll
    for (int h = 0; h < FPT; ++h) t[h] = act[h] ? my[h].t + 1 : 0;
    bool later = false;  // some frame of the group is past its first sweep
#pragma unroll
    for (int h = 0; h < FPT; ++h) later |= t[h] > 1;
    bool halted = false;
    sweep_rows<FPT, CH, DB, WIN, SELFLAST>(p.mb, any, s_rptr, s_spe, z, Z, later, t, xlo, tab,
                                           QP, SV, S, R, bar_id, bar_n, p.edges, bits, wst,
                                           okb, M, halted);
    bool done[FPT], full[FPT];
#pragma unroll
    for (int h = 0; h < FPT; ++h) full[h] = false;
    if constexpr (WIN) {
      // Step 3: the hard decisions of the latest V2C phase; iters = the sweep in which
      // the window filled, negated when it never did
      done[0] = act[0] && (halted || t[0] >= p.max_iter);
      if (done[0]) {
        uint32_t* ho = p.hard + static_cast<long long>(frame[0]) * words;
        for (int w = z; w < words; w += Z) ho[w] = bits[w];
        if (z == 0) p.iters[frame[0]] = halted ? t[0] : -t[0];
      }
      team_sync(bar_id, bar_n);
      if (done[0])
        for (int w = z; w < wpad; w += Z) bits[w] = 0u;  // ready for the slot's next frame
    } else {
      // ---- end of the sweep: flushed posterior (Eq. s4e20 read-only), hard decisions
      // (Eq. s2e7) and the syndrome stop.  A frame stops only when every check holds, so
      // the checks of one base row (the test row) are evaluated first; when one of them
      // fails, the frame goes on and the full flush and syndrome scan are skipped (the
      // syndrome is non-zero whatever the other rows give: the same decision).
      if (lane && z == 0)
  #pragma unroll
        for (int h = 0; h < FPT; ++h) my[h].unsat = 0;
      team_sync(bar_id, bar_n);
      if (p.stop == CBP_STOP_SYNDROME && any) {
        bool test[FPT];
        bool tany = false;
  #pragma unroll
        for (int h = 0; h < FPT; ++h) {
          test[h] = act[h] && t[h] < p.max_iter;
          tany |= test[h];
        }
        if (tany) {
          uint32_t par[FPT];
  #pragma unroll
          for (int h = 0; h < FPT; ++h) par[h] = 0;
          test_row_parity<FPT>(p, s_rptr, s_col, z, Z, xlo, tab, QP, SV, S, par);
  #pragma unroll
          for (int h = 0; h < FPT; ++h)
            if (test[h] && par[h]) my[h].unsat = 1;
        }
      }
      team_sync(bar_id, bar_n);
      bool any_full = false;
  #pragma unroll
      for (int h = 0; h < FPT; ++h) {
        full[h] = act[h] && (t[h] >= p.max_iter ||
                             (p.stop == CBP_STOP_SYNDROME &&
                              *static_cast<volatile int*>(&my[h].unsat) == 0));
        any_full |= full[h];
      }
      // the decision bits of every frame are zero here (cleared at the start and after
      // each full test); the warp skips the flush when none of its frames needs it
      if (__any_sync(0xffffffffu, any_full)) {
        for (int c = 0; c < p.nb; ++c) {
          const uint2 ci = s_col[c];
          const int idx = ci.y & 0xffff;
          const int sk = int(ci.x >> 16), rk = int(ci.x & 0xffff);
          float qv[FPT], pv[FPT], Sk[FPT];
          int v = 0;
          if (any_full) {
            if (ci.y & 0x10000u) {  // weight-1 column: lane z owns its single check (rk, z)
              LV::ld_pair(SV, idx * Z + z, qv, pv);
              LV::ld(S, rk * Z + z, Sk);
              v = c * Z + mod_add(z + sk, Z);
            } else {
              LV::ld_pair(QP, idx * Z + z, qv, pv);
              int zk = z - sk;
              zk = zk < 0 ? zk + Z : zk;
              LV::ld(S, rk * Z + zk, Sk);
              v = c * Z + z;
            }
          }
  #pragma unroll
          for (int h = 0; h < FPT; ++h) {
            bool neg = false;
            if (full[h]) {
              const float mag = phi_eval(fabsf(__fsub_rn(fabsf(Sk[h]), pv[h])), xlo, tab);
              const float lb = __fadd_rn(
                  qv[h], __uint_as_float(__float_as_uint(mag) |
                                         ((__float_as_uint(Sk[h]) ^ __float_as_uint(qv[h])) &
                                          0x80000000u)));
              neg = lb < 0.0f;
              if (p.soft) p.soft[static_cast<long long>(frame[h]) * N + v] = lb;
            }
            if (words_aligned) {
              // Z % 32 == 0: a warp lies inside one lane group, and its 32 variables of
              // column c are 32 consecutive positions of the column (rotated by the shift
              // for a weight-1 column), i.e. one aligned word or two partial ones
              const unsigned wv = __ballot_sync(0xffffffffu, neg);
              if ((tid & 31) == 0 && full[h]) {
                uint32_t* wb = bits + h * wpad;
                const int p0 = v - c * Z;  // position of this lane's variable in column c
                const int sh = p0 & 31;
                if (sh == 0) {
                  wb[v >> 5] = wv;  // the word holds exactly this warp's variables
                } else {
                  atomicOr(wb + (v >> 5), wv << sh);
                  atomicOr(wb + ((c * Z + mod_add(p0 - sh + 32, Z)) >> 5), wv >> (32 - sh));
                }
              }
            } else {
              warp_or_bit(bits + h * wpad + (v >> 5), neg ? (1u << (v & 31)) : 0u, full[h]);
            }
          }
        }
      }
      team_sync(bar_id, bar_n);
      // ---- syndrome of the frames tested in full; a frame stops scanning once one of
      // its checks is unsatisfied
      if (any_full) {
        bool open[FPT];
        bool scan = false;
  #pragma unroll
        for (int h = 0; h < FPT; ++h) {
          open[h] = full[h];
          scan |= open[h];
        }
        for (int r = 0; r < p.mb && scan; ++r) {
          uint32_t pr[FPT];
  #pragma unroll
          for (int h = 0; h < FPT; ++h) pr[h] = 0;
          for (int k = s_rptr[r]; k < s_rptr[r + 1]; ++k) {
            const BaseEdge be = p.edges[k];  // read through L1: the scan is off the hot path
            const int v = be.c * Z + mod_add(z + be.s, Z);
  #pragma unroll
            for (int h = 0; h < FPT; ++h) pr[h] ^= bits[h * wpad + (v >> 5)] >> (v & 31);
          }
          scan = false;
  #pragma unroll
          for (int h = 0; h < FPT; ++h) {
            if (open[h] && (pr[h] & 1u)) my[h].unsat = 1;
            open[h] = open[h] && !*static_cast<volatile int*>(&my[h].unsat);
            scan |= open[h];
          }
        }
      }
      team_sync(bar_id, bar_n);
  #pragma unroll
      for (int h = 0; h < FPT; ++h) {
        done[h] = false;
        if (full[h]) {
          const bool ok = my[h].unsat == 0;
          done[h] = (ok && p.stop == CBP_STOP_SYNDROME) || t[h] >= p.max_iter;
          if (done[h]) {
            uint32_t* ho = p.hard + static_cast<long long>(frame[h]) * words;
            for (int w = z; w < words; w += Z) ho[w] = bits[h * wpad + w];
            if (z == 0) p.iters[frame[h]] = ok ? t[h] : -t[h];
          }
        }
      }
    }  // not WIN
    team_sync(bar_id, bar_n);
    if constexpr (!WIN) {
  #pragma unroll
      for (int h = 0; h < FPT; ++h)  // ready for the next full test
        if (full[h])
          for (int w = z; w < words; w += Z) bits[h * wpad + w] = 0u;
    }
    if (z == 0) {
#pragma unroll
      for (int h = 0; h < FPT; ++h)
        if (act[h]) {
          if (done[h]) {
            my[h].frame = frame[h] + stride;
            my[h].t = 0;
          } else {
            my[h].t = t[h];
          }
        }
    }
    team_sync(bar_id, bar_n);
  }
}

template <bool CHKS, int FPT, int CH, bool DB, int MAXT, bool SELFLAST = false>
__global__ void __launch_bounds__(MAXT, 1) cbp_sp_kernel(const KParams p) {
  extern __shared__ __align__(16) unsigned char smem[];
  sp_body<CHKS, FPT, CH, DB, false, SELFLAST>(p, blockIdx.x * p.F * FPT, p.slots, p.batch,
                                               smem, true);
}

// The paper-literal stop of Eq. (s4e24) with the Step 3 output (one frame per group).
template <bool CHKS>
__global__ void __launch_bounds__(768, 1) cbp_sp_win_kernel(const KParams p) {
  extern __shared__ __align__(16) unsigned char smem[];
  sp_body<CHKS, 1, 4, false, true>(p, blockIdx.x * p.F, p.slots, p.batch, smem, true);
}

// Several codes in one persistent launch: each CTA takes chunks (code, frame range) from
// a work counter, in the order of the segment list, and decodes them with that code's
// lane-group layout.
template <bool CHKS, int FPT, int CH, bool DB, int MAXT, bool SELFLAST = false>
__global__ void __launch_bounds__(MAXT, 1) cbp_sp_multi_kernel(const MultiParams mp) {
  extern __shared__ __align__(16) unsigned char smem[];
  // the chunk's code parameters live in shared memory (read like kernel parameters)
  __shared__ KParams s_p;
  __shared__ int s_chunk[2];  // chunk index, frame range start
  const int total = mp.seg_end[mp.nseg - 1];
  for (bool first_chunk = true;; first_chunk = false) {
    if (threadIdx.x == 0) {
      const int c = atomicAdd(mp.counter, 1);
      s_chunk[0] = c;
      if (c < total) {
        int k = 0;
        while (c >= mp.seg_end[k]) ++k;
        s_p = mp.code[mp.seg_code[k]];
        s_chunk[1] = mp.seg_frame0[k] + (k == 0 ? c : c - mp.seg_end[k - 1]) * mp.seg_frames[k];
        s_p.batch = min(s_chunk[1] + mp.seg_frames[k], mp.seg_frame1[k]);  // range end
      }
    }
    __syncthreads();
    if (s_chunk[0] >= total) break;
    sp_body<CHKS, FPT, CH, DB, false, SELFLAST>(s_p, s_chunk[1], s_p.F * FPT, s_p.batch, smem,
                                               first_chunk);
    __syncthreads();
  }
}

}  // namespace

void* sp_multi_kernel_ptr(bool chk_shared, int fpt, bool self_last) {
  if (fpt == 2)
    return chk_shared ? reinterpret_cast<void*>(&cbp_sp_multi_kernel<true, 2, 4, true, 384>)
                      : reinterpret_cast<void*>(&cbp_sp_multi_kernel<false, 2, 4, true, 384>);
  if (self_last)  // every item's code ends its rows with the weight-1 edge
    return chk_shared
               ? reinterpret_cast<void*>(&cbp_sp_multi_kernel<true, 1, 3, false, 768, true>)
               : reinterpret_cast<void*>(&cbp_sp_multi_kernel<false, 1, 3, false, 768, true>);
  return chk_shared ? reinterpret_cast<void*>(&cbp_sp_multi_kernel<true, 1, 4, false, 768>)
                    : reinterpret_cast<void*>(&cbp_sp_multi_kernel<false, 1, 4, false, 768>);
}

void* sp_win_kernel_ptr(bool chk_shared) {
  return chk_shared ? reinterpret_cast<void*>(&cbp_sp_win_kernel<true>)
                    : reinterpret_cast<void*>(&cbp_sp_win_kernel<false>);
}

void* sp_kernel_ptr(bool chk_shared, int fpt, bool wide, bool self_last) {
  // wide: up to 1024 threads per CTA (Z > 512), fewer registers per thread
  if (wide)
    return chk_shared ? reinterpret_cast<void*>(&cbp_sp_kernel<true, 1, 2, true, 1024>)
                      : reinterpret_cast<void*>(&cbp_sp_kernel<false, 1, 2, true, 1024>);
  if (fpt == 2)
    return chk_shared ? reinterpret_cast<void*>(&cbp_sp_kernel<true, 2, 4, true, 384>)
                      : reinterpret_cast<void*>(&cbp_sp_kernel<false, 2, 4, true, 384>);
  // one frame per lane group, up to 768 threads: two 384-lane teams per CTA progress
  // independently and hide each other's memory latency
  if (self_last)  // chunks of 3 measured best once whole chunks run unguarded
    return chk_shared ? reinterpret_cast<void*>(&cbp_sp_kernel<true, 1, 3, false, 768, true>)
                      : reinterpret_cast<void*>(&cbp_sp_kernel<false, 1, 3, false, 768, true>);
  return chk_shared ? reinterpret_cast<void*>(&cbp_sp_kernel<true, 1, 4, false, 768>)
                    : reinterpret_cast<void*>(&cbp_sp_kernel<false, 1, 4, false, 768>);
}

}  // namespace cbp
