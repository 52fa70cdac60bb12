// CBP, log-tanh form (Sec. IV-C, Steps 1-3), on a wavefront schedule of the expanded
// Tanner graph: the kernel for codes with small lifting sizes (down to Z = 1, codes given
// as plain parity-check matrices such as PEG codes), where the Z checks of a base row are
// too few to fill the lanes of the lane-parallel kernel.
//
// The paper's order visits the checks m = 0, 1, ..., M-1 one after another.  A check only
// depends on the checks before it that share one of its variables (it reads their
// (Q*, phi) and check-beliefs and writes their C2V slots).  The host gives every check the
// level 1 + max(level of the previous check of each of its variables), 0 if none, so the
// checks of one level share no variable and none is another's predecessor.  Running the
// levels in order, each level's checks in any order, gives every check exactly the inputs
// it has in the sequential order: the result is that order's, bit for bit.  (A QC code's
// base row is such a level; a random PEG code with N = 2048 has 24 levels per sweep.)
//
// A CTA holds F lane groups of G lanes (whole warps); each group decodes one frame at a
// time.  Lane l takes the checks l, l + G, ... of a level; a named barrier over the group
// ends the level.  Checks are numbered in level order (ci).  Per group, shared memory
// holds the frame's state:
//   Q    Q*_v for every variable (phi(|Q*_v|) is evaluated where it is read: keeping only
//        Q* leaves room for more frames per SM)                       [N]
//   S    check-beliefs, sign bit = sgn Omega, by level-ordered check  [M]
//   bits decisions of the flushed posterior                          [words]
// and the workspace the C2V messages R, indexed by the level-ordered edge, so the own
// slots of a check are contiguous.  Level-ordered tables (host-built):
//   lvl_ptr  [L + 1]  level l holds the checks [lvl_ptr[l], lvl_ptr[l + 1])
//   lvl_e0   [M + 1]  first edge of each check; the next entry ends it
//   lvl_edge [E]      (v | first << 30 | self << 31, predecessor check, predecessor edge)
//   lvl_rec8 [E]      the same in 8 bytes (v | flags, predecessor edge | check << 20), when
//                     M <= 4096 and E < 2^20; SHREC instances copy it and lvl_e0 into
//                     shared memory instead of reading lvl_edge through L1
//   last_chk [N]      the last check of each variable (flushed posterior)
// The per-edge arithmetic is the lane-parallel kernel's, operation for operation.
#include "cbp_kernel_common.cuh"

namespace cbp {
namespace {

constexpr int kLvlChunk = 3;        // edges of a check whose loads are issued together
constexpr int kLvlMaxThreads = 768;

// One edge record: variable and flags, predecessor check, predecessor edge.
struct LvlRec {
  uint32_t vx;
  int cj, pe;
};

template <bool SHREC>
__device__ __forceinline__ LvlRec lvl_rec(const uint2* s_rec, const LvlEdge* __restrict__ led,
                                          int e) {
  LvlRec r;
  if (SHREC) {
    const uint2 a = s_rec[e];
    r.vx = a.x;
    r.cj = static_cast<int>(a.y >> 20);
    r.pe = static_cast<int>(a.y & 0xFFFFFu);
  } else {
    const uint4 a = __ldg(led + e);
    r.vx = a.x;
    r.cj = static_cast<int>(a.y);
    r.pe = static_cast<int>(a.z);
  }
  return r;
}

template <bool SHREC>
__global__ void __launch_bounds__(kLvlMaxThreads, 1) cbp_level_kernel(const KParams p) {
  extern __shared__ __align__(16) unsigned char smem[];
  const int G = p.lvl_lanes, F = p.F;
  const int N = p.N, M = p.M, E = p.E, words = p.words;
  const int tid = threadIdx.x;
  const int g = tid / G, l = tid - g * G;
  unsigned char* sp = smem;
  float4* s_tab = reinterpret_cast<float4*>(sp);
  sp += sizeof(float4) * kPhiSegments;
  int* s_unsat = reinterpret_cast<int*>(sp);  // per group: a check of the frame fails
  sp += sizeof(int) * 16;
  uint2* s_rec = reinterpret_cast<uint2*>(sp);
  int* s_e0 = reinterpret_cast<int*>(sp + sizeof(uint2) * E);
  if (SHREC) sp += sizeof(uint2) * E + sizeof(int) * ((M + 1 + 3) & ~3);
  for (int i = tid; i < kPhiSegments; i += blockDim.x) s_tab[i] = p.phi_tab[i];
  if (tid < 16) s_unsat[tid] = 0;
  if (SHREC) {
    for (int i = tid; i < E; i += blockDim.x) s_rec[i] = p.lvl_rec8[i];
    for (int i = tid; i <= M; i += blockDim.x) s_e0[i] = p.lvl_e0[i];
  }
  __syncthreads();
  if (g >= F) return;
  const int* e0t = SHREC ? s_e0 : p.lvl_e0;
  const LvlEdge* __restrict__ led = p.lvl_edge;
  float* gb = reinterpret_cast<float*>(sp) + static_cast<size_t>(g) * p.sh_frame;
  float* Qv = gb;
  float* S = gb + ((N + 3) & ~3);
  uint32_t* bits = reinterpret_cast<uint32_t*>(S + ((M + 3) & ~3));
  const long long slot = static_cast<long long>(blockIdx.x) * F + g;
  float* R = p.ws + slot * p.ws_slot;
  const float4* tab = s_tab;
  const float xlo = p.phi_xlo;
  const int bar_id = 1 + g;

  for (long long frame = slot; frame < p.batch; frame += p.slots) {
    // ---- Step 1, Eq. (s4e15): Q*_v = L_v (+0 turns -0 into +0)
    const float* src = p.llr + frame * N;
    bool bad = false;
    for (int v = l; v < N; v += G) {
      const float L = __fadd_rn(__ldg(src + v), 0.0f);
      bad |= non_finite(L);
      Qv[v] = L;
    }
    if (bad) atomicOr(p.status, kStatusNonFiniteLlr);
    team_sync(bar_id, G);

    for (int t = 1;; ++t) {
      // ---- Step 2: the levels in order, a level's checks on the lanes
      for (int lv = 0; lv < p.nlev; ++lv) {
        const int i1 = p.lvl_ptr[lv + 1];
        for (int ci = p.lvl_ptr[lv] + l; ci < i1; ci += G) {
          const int e1 = e0t[ci + 1];
          float Sacc = 0.0f;
          uint32_t sig = 0;
          for (int eb = e0t[ci]; eb < e1; eb += kLvlChunk) {
            float q[kLvlChunk], sj[kLvlChunk], ro[kLvlChunk];
            uint32_t vx[kLvlChunk];
            int pe[kLvlChunk];
#pragma unroll
            for (int j = 0; j < kLvlChunk; ++j) {  // loads of the chunk
              const int e = eb + j;
              if (e < e1) {
                const LvlRec rec = lvl_rec<SHREC>(s_rec, led, e);
                vx[j] = rec.vx;
                pe[j] = rec.pe;
                q[j] = Qv[rec.vx & kSpMask];
                sj[j] = S[rec.cj];
                ro[j] = (!(rec.vx & kSpSelf) && t > 1) ? R[e] : 0.0f;
              }
            }
#pragma unroll
            for (int j = 0; j < kLvlChunk; ++j) {  // the updates, in column order
              if (eb + j < e1) {
                const bool self = vx[j] & kSpSelf;
                // B2V, Eqs. (s4e18), (s4e13); a variable not visited before adds no C2V
                // phi(|Q*_v|) of Eq. (s4e18), the value C2B stored with Q*_v
                const float phq = phi_eval(fabsf(q[j]), xlo, tab);
                const float mag = phi_eval(fabsf(__fsub_rn(fabsf(sj[j]), phq)), xlo, tab);
                const float rb = __uint_as_float(
                    __float_as_uint(mag) |
                    ((__float_as_uint(sj[j]) ^ __float_as_uint(q[j])) & 0x80000000u));
                const bool first = (t == 1) && (vx[j] & kSpFirst);
                const float Rn = first ? 0.0f : rb;
                // V2C, Eqs. (s4e20), (s4e19); weight-1 column: c_j == c_i
                const float rold = self ? Rn : ro[j];
                const float qn = __fsub_rn(__fadd_rn(q[j], Rn), rold);
                // C2B, Eq. (s4e21) as a sum of phi; the sign bits fold into sig
                const float phn = phi_eval(fabsf(qn), xlo, tab);
                Sacc = __fadd_rn(Sacc, phn);
                sig ^= __float_as_uint(qn);
                if (!self && !first) R[pe[j]] = Rn;  // R_{c_j->v} <- R^new, Eq. (s4e22)
                Qv[vx[j] & kSpMask] = qn;
              }
            }
          }
          // Eq. (s4e23); the sign bit carries sgn(Omega)
          S[ci] = __uint_as_float(__float_as_uint(Sacc) | (sig & 0x80000000u));
        }
        team_sync(bar_id, G);
      }
      // ---- sweep-end test: a frame stops only when every check holds, so the checks of
      // the widest level are evaluated first (on the read-only flushed posterior); when one
      // fails, the full flush and syndrome are skipped (the same decision)
      bool full = t >= p.max_iter;
      if (!full && p.stop == CBP_STOP_SYNDROME) {
        bool fail = false;
        const int j1 = p.lvl_ptr[p.lvl_test + 1];
        for (int ci = p.lvl_ptr[p.lvl_test] + l; ci < j1; ci += G) {
          uint32_t par = 0;
          const int e1 = e0t[ci + 1];
          for (int e = e0t[ci]; e < e1; ++e) {
            const int v = static_cast<int>(lvl_rec<SHREC>(s_rec, led, e).vx & kSpMask);
            const float2 qp = make_float2(Qv[v], phi_eval(fabsf(Qv[v]), xlo, tab));
            const float Sk = S[__ldg(p.last_chk + v)];
            const float mag = phi_eval(fabsf(__fsub_rn(fabsf(Sk), qp.y)), xlo, tab);
            const float lb = __fadd_rn(
                qp.x, __uint_as_float(__float_as_uint(mag) |
                                      ((__float_as_uint(Sk) ^ __float_as_uint(qp.x)) &
                                       0x80000000u)));
            par ^= lb < 0.0f ? 1u : 0u;
          }
          fail |= (par & 1u) != 0;
        }
        if (fail) s_unsat[g] = 1;
        team_sync(bar_id, G);
        full = *static_cast<volatile int*>(&s_unsat[g]) == 0;
        team_sync(bar_id, G);
        if (l == 0) s_unsat[g] = 0;
      }
      if (!full) continue;
      // ---- flushed posterior (Eq. s4e20 with the last check of v, read-only) and the
      // decisions (Eq. s2e7): lane l takes v = l, l + G, ...; a warp's 32 variables of one
      // step are one aligned word
      for (int vb = 0; vb < N; vb += G) {
        const int v = vb + l;
        bool neg = false;
        if (v < N) {
          const float2 qp = make_float2(Qv[v], phi_eval(fabsf(Qv[v]), xlo, tab));
          const float Sk = S[__ldg(p.last_chk + v)];
          const float mag = phi_eval(fabsf(__fsub_rn(fabsf(Sk), qp.y)), xlo, tab);
          const float lb = __fadd_rn(
              qp.x, __uint_as_float(__float_as_uint(mag) |
                                    ((__float_as_uint(Sk) ^ __float_as_uint(qp.x)) &
                                     0x80000000u)));
          neg = lb < 0.0f;
          if (p.soft) p.soft[frame * N + v] = lb;
        }
        const unsigned wv = __ballot_sync(0xffffffffu, neg);
        if ((l & 31) == 0 && v < N) bits[v >> 5] = wv;
      }
      team_sync(bar_id, G);
      // ---- syndrome: every check's parity over its variables' decisions
      bool fail = false;
      for (int ci = l; ci < M; ci += G) {
        uint32_t par = 0;
        const int e1 = e0t[ci + 1];
        for (int e = e0t[ci]; e < e1; ++e) {
          const uint32_t v = lvl_rec<SHREC>(s_rec, led, e).vx & kSpMask;
          par ^= bits[v >> 5] >> (v & 31);
        }
        fail |= (par & 1u) != 0;
      }
      if (fail) s_unsat[g] = 1;
      team_sync(bar_id, G);
      const bool ok = *static_cast<volatile int*>(&s_unsat[g]) == 0;
      const bool done = (ok && p.stop == CBP_STOP_SYNDROME) || t >= p.max_iter;
      if (done) {  // Step 3
        uint32_t* ho = p.hard + frame * words;
        for (int w = l; w < words; w += G) ho[w] = bits[w];
        if (l == 0) p.iters[frame] = ok ? t : -t;
      }
      team_sync(bar_id, G);
      if (l == 0) s_unsat[g] = 0;
      team_sync(bar_id, G);
      if (done) break;
    }
  }
}

// Layered normalized min-sum (Eqs. s2e10, s2e12), the comparator, on the same wavefront
// schedule: a check reads and writes only its variables' Lambda and its own state, so the
// levels order it exactly as the sequential schedule does.  Per group, shared memory
// holds the check states (min1 | sgn, min2, position of min1, 32 sign bits) by
// level-ordered check, Lambda for every variable and the decision bits; SHV instances
// also copy each edge's variable index and the check offsets into shared memory.  The
// arithmetic is the lane-parallel layered kernel's, operation for operation: pass 1 forms
// Q = Lambda - R_old and the minima, pass 2 forms Q again from the same Lambda and R_old
// (the same rounding) and Lambda = Q + R_new.
constexpr int kLbpChunk = 4;
constexpr float kLvlInf = __builtin_huge_valf();

template <bool SHV>
__global__ void __launch_bounds__(kLvlMaxThreads, 1) lbp_level_kernel(const KParams p) {
  extern __shared__ __align__(16) unsigned char smem[];
  const int G = p.lvl_lanes, F = p.F;
  const int N = p.N, M = p.M, E = p.E, words = p.words;
  const int tid = threadIdx.x;
  const int g = tid / G, l = tid - g * G;
  const float alpha = p.alpha;
  unsigned char* sp = smem;
  int* s_unsat = reinterpret_cast<int*>(sp);
  sp += sizeof(int) * 16;
  uint32_t* s_v = reinterpret_cast<uint32_t*>(sp);
  int* s_e0 = reinterpret_cast<int*>(sp + sizeof(uint32_t) * ((E + 3) & ~3));
  if (SHV) sp += sizeof(uint32_t) * ((E + 3) & ~3) + sizeof(int) * ((M + 1 + 3) & ~3);
  if (tid < 16) s_unsat[tid] = 0;
  if (SHV) {
    for (int i = tid; i < E; i += blockDim.x) s_v[i] = p.lvl_edge[i].x & kSpMask;
    for (int i = tid; i <= M; i += blockDim.x) s_e0[i] = p.lvl_e0[i];
  }
  __syncthreads();
  if (g >= F) return;
  const int* e0t = SHV ? s_e0 : p.lvl_e0;
  const LvlEdge* __restrict__ led = p.lvl_edge;
  float* gb = reinterpret_cast<float*>(sp) + static_cast<size_t>(g) * p.sh_frame;
  uint4* AUX = reinterpret_cast<uint4*>(gb);
  float* VAR = gb + 4 * static_cast<size_t>(M);
  uint32_t* bits = reinterpret_cast<uint32_t*>(VAR + ((N + 3) & ~3));
  const long long slot = static_cast<long long>(blockIdx.x) * F + g;
  const int bar_id = 1 + g;
  auto var_of = [&](int e) -> int {
    return SHV ? static_cast<int>(s_v[e]) : static_cast<int>(__ldg(&led[e].x) & kSpMask);
  };

  for (long long frame = slot; frame < p.batch; frame += p.slots) {
    const float* src = p.llr + frame * N;
    bool bad = false;
    for (int v = l; v < N; v += G) {  // Lambda_v = L_v (+0 turns -0 into +0)
      const float L = __fadd_rn(__ldg(src + v), 0.0f);
      bad |= non_finite(L);
      VAR[v] = L;
    }
    if (bad) atomicOr(p.status, kStatusNonFiniteLlr);
    team_sync(bar_id, G);

    for (int t = 1;; ++t) {
      for (int lv = 0; lv < p.nlev; ++lv) {
        const int i1 = p.lvl_ptr[lv + 1];
        for (int ci = p.lvl_ptr[lv] + l; ci < i1; ci += G) {
          const int k0 = e0t[ci], d = e0t[ci + 1] - k0;
          float r1 = 0.0f, r2 = 0.0f;
          uint32_t osig = 0, oidx = 0, osg = 0;
          if (t > 1) {  // rebuild R_old from the check's state of the previous sweep
            const uint4 a = AUX[ci];
            r1 = __fmul_rn(alpha, fabsf(__uint_as_float(a.x)));
            r2 = __fmul_rn(alpha, __uint_as_float(a.y));
            osig = a.x >> 31;
            oidx = a.z;
            osg = a.w;
          }
          float m1 = kLvlInf, m2 = kLvlInf;
          uint32_t idx = 0, sig = 0, sg = 0;
          for (int j0 = 0; j0 < d; j0 += kLbpChunk) {  // pass 1, Eq. (s2e10)
            float lam[kLbpChunk];
#pragma unroll
            for (int u = 0; u < kLbpChunk; ++u)
              if (j0 + u < d) lam[u] = VAR[var_of(k0 + j0 + u)];
#pragma unroll
            for (int u = 0; u < kLbpChunk; ++u) {
              const int j = j0 + u;
              if (j < d) {
                float rold = 0.0f;
                if (t > 1) {
                  const float rm = (static_cast<uint32_t>(j) == oidx) ? r2 : r1;
                  rold = (osig ^ ((osg >> j) & 1u)) ? -rm : rm;
                }
                const float q = __fsub_rn(lam[u], rold);
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
          }
          const float n1 = __fmul_rn(alpha, m1), n2 = __fmul_rn(alpha, m2);
          for (int j0 = 0; j0 < d; j0 += kLbpChunk) {  // pass 2, Eq. (s2e12)
            float lam[kLbpChunk];
            int vv[kLbpChunk];
#pragma unroll
            for (int u = 0; u < kLbpChunk; ++u)
              if (j0 + u < d) {
                vv[u] = var_of(k0 + j0 + u);
                lam[u] = VAR[vv[u]];
              }
#pragma unroll
            for (int u = 0; u < kLbpChunk; ++u) {
              const int j = j0 + u;
              if (j < d) {
                float rold = 0.0f;
                if (t > 1) {
                  const float rm = (static_cast<uint32_t>(j) == oidx) ? r2 : r1;
                  rold = (osig ^ ((osg >> j) & 1u)) ? -rm : rm;
                }
                const float q = __fsub_rn(lam[u], rold);
                const float rm = (static_cast<uint32_t>(j) == idx) ? n2 : n1;
                VAR[vv[u]] = __fadd_rn(q, (sig ^ ((sg >> j) & 1u)) ? -rm : rm);
              }
            }
          }
          AUX[ci] = make_uint4(__float_as_uint(sig ? -m1 : m1), __float_as_uint(m2), idx, sg);
        }
        team_sync(bar_id, G);
      }
      // ---- sweep-end test: a frame stops only when every check holds, so the checks of
      // the widest level are evaluated first (on the read-only flushed posterior); when one
      // fails, the full flush and syndrome are skipped (the same decision)
      bool full = t >= p.max_iter;
      if (!full && p.stop == CBP_STOP_SYNDROME) {
        bool fail = false;
        const int j1 = p.lvl_ptr[p.lvl_test + 1];
        for (int ci = p.lvl_ptr[p.lvl_test] + l; ci < j1; ci += G) {
          uint32_t par = 0;
          const int e1 = e0t[ci + 1];
          for (int e = e0t[ci]; e < e1; ++e) {
            const int v = var_of(e);
            const float lb = VAR[v];
            par ^= lb < 0.0f ? 1u : 0u;
          }
          fail |= (par & 1u) != 0;
        }
        if (fail) s_unsat[g] = 1;
        team_sync(bar_id, G);
        full = *static_cast<volatile int*>(&s_unsat[g]) == 0;
        team_sync(bar_id, G);
        if (l == 0) s_unsat[g] = 0;
      }
      if (!full) continue;
      // ---- decisions (Eq. s2e7) on Lambda, packed by warp ballot; syndrome
      for (int vb = 0; vb < N; vb += G) {
        const int v = vb + l;
        bool neg = false;
        if (v < N) {
          const float lb = VAR[v];
          neg = lb < 0.0f;
          if (p.soft) p.soft[frame * N + v] = lb;
        }
        const unsigned wv = __ballot_sync(0xffffffffu, neg);
        if ((l & 31) == 0 && v < N) bits[v >> 5] = wv;
      }
      team_sync(bar_id, G);
      bool fail = false;
      for (int ci = l; ci < M; ci += G) {
        uint32_t par = 0;
        const int e1 = e0t[ci + 1];
        for (int e = e0t[ci]; e < e1; ++e) {
          const uint32_t v = static_cast<uint32_t>(var_of(e));
          par ^= bits[v >> 5] >> (v & 31);
        }
        fail |= (par & 1u) != 0;
      }
      if (fail) s_unsat[g] = 1;
      team_sync(bar_id, G);
      const bool ok = *static_cast<volatile int*>(&s_unsat[g]) == 0;
      const bool done = (ok && p.stop == CBP_STOP_SYNDROME) || t >= p.max_iter;
      if (done) {
        uint32_t* ho = p.hard + frame * words;
        for (int w = l; w < words; w += G) ho[w] = bits[w];
        if (l == 0) p.iters[frame] = ok ? t : -t;
      }
      team_sync(bar_id, G);
      if (l == 0) s_unsat[g] = 0;
      team_sync(bar_id, G);
      if (done) break;
    }
  }
}

// CBP normalized min-sum (Eqs. s4e18xx, s4e21xx) on the same schedule and tables: the
// log-tanh kernel's structure with the check state (min1 | sgn Omega, min2) in place of
// the check-belief and Q* alone per variable; the C2V messages per edge in the workspace
// (B2V writes the predecessor's slot, V2C reads the edge's own slot).  The arithmetic is
// the lane-parallel CBP min-sum kernel's with per-edge messages, operation for operation.
template <bool SHREC>
__global__ void __launch_bounds__(kLvlMaxThreads, 1) nms_level_kernel(const KParams p) {
  extern __shared__ __align__(16) unsigned char smem[];
  const int G = p.lvl_lanes, F = p.F;
  const int N = p.N, M = p.M, E = p.E, words = p.words;
  const int tid = threadIdx.x;
  const int g = tid / G, l = tid - g * G;
  const float alpha = p.alpha;
  unsigned char* sp = smem;
  int* s_unsat = reinterpret_cast<int*>(sp);
  sp += sizeof(int) * 16;
  uint2* s_rec = reinterpret_cast<uint2*>(sp);
  int* s_e0 = reinterpret_cast<int*>(sp + sizeof(uint2) * E);
  if (SHREC) sp += sizeof(uint2) * E + sizeof(int) * ((M + 1 + 3) & ~3);
  if (tid < 16) s_unsat[tid] = 0;
  if (SHREC) {
    for (int i = tid; i < E; i += blockDim.x) s_rec[i] = p.lvl_rec8[i];
    for (int i = tid; i <= M; i += blockDim.x) s_e0[i] = p.lvl_e0[i];
  }
  __syncthreads();
  if (g >= F) return;
  const int* e0t = SHREC ? s_e0 : p.lvl_e0;
  const LvlEdge* __restrict__ led = p.lvl_edge;
  float* gb = reinterpret_cast<float*>(sp) + static_cast<size_t>(g) * p.sh_frame;
  float2* CHK = reinterpret_cast<float2*>(gb);
  float* Q = gb + 2 * static_cast<size_t>(M);
  uint32_t* bits = reinterpret_cast<uint32_t*>(Q + ((N + 3) & ~3));
  const long long slot = static_cast<long long>(blockIdx.x) * F + g;
  float* R = p.ws + slot * p.ws_slot;
  const int bar_id = 1 + g;

  for (long long frame = slot; frame < p.batch; frame += p.slots) {
    const float* src = p.llr + frame * N;
    bool bad = false;
    for (int v = l; v < N; v += G) {  // Q*_v = L_v (+0 turns -0 into +0)
      const float L = __fadd_rn(__ldg(src + v), 0.0f);
      bad |= non_finite(L);
      Q[v] = L;
    }
    if (bad) atomicOr(p.status, kStatusNonFiniteLlr);
    team_sync(bar_id, G);

    for (int t = 1;; ++t) {
      for (int lv = 0; lv < p.nlev; ++lv) {
        const int i1 = p.lvl_ptr[lv + 1];
        for (int ci = p.lvl_ptr[lv] + l; ci < i1; ci += G) {
          const int e0 = e0t[ci], e1 = e0t[ci + 1];
          float m1 = kLvlInf, m2 = kLvlInf;
          uint32_t sig = 0;
          for (int eb = e0; eb < e1; eb += kLbpChunk) {
            float q[kLbpChunk], ro[kLbpChunk];
            float2 pc[kLbpChunk];
            uint32_t vx[kLbpChunk];
            int pe[kLbpChunk];
#pragma unroll
            for (int u = 0; u < kLbpChunk; ++u) {  // loads of the chunk
              const int e = eb + u;
              if (e < e1) {
                const LvlRec rec = lvl_rec<SHREC>(s_rec, led, e);
                vx[u] = rec.vx;
                pe[u] = rec.pe;
                q[u] = Q[rec.vx & kSpMask];
                pc[u] = CHK[rec.cj];
                ro[u] = (t > 1 && !(rec.vx & kSpSelf)) ? R[e] : 0.0f;
              }
            }
#pragma unroll
            for (int u = 0; u < kLbpChunk; ++u) {
              const int e = eb + u;
              if (e < e1) {
                const bool self = vx[u] & kSpSelf;
                const bool first = (t == 1) && (vx[u] & kSpFirst);
                // B2V, Eq. (s4e18xx): min2 of c_j when |Q*_v| is its min1
                float Rn = 0.0f;
                if (!first) {
                  const float b1 = fabsf(pc[u].x);
                  const float rm = __fmul_rn(alpha, (fabsf(q[u]) == b1) ? pc[u].y : b1);
                  Rn = (sign_bit(pc[u].x) ^ (q[u] < 0.0f)) ? -rm : rm;
                }
                float rold;
                if (self) {
                  rold = Rn;  // c_j == c_i
                } else {
                  rold = ro[u];
                  if (!first) R[pe[u]] = Rn;  // Eq. (s4e22)
                }
                const float qn = __fsub_rn(__fadd_rn(q[u], Rn), rold);  // Eq. (s4e19)
                const float a = fabsf(qn);                                 // C2B, Eq. (s4e21xx)
                if (a < m1) {
                  m2 = m1;
                  m1 = a;
                } else if (a < m2) {
                  m2 = a;
                }
                sig ^= qn < 0.0f;
                Q[vx[u] & kSpMask] = qn;
              }
            }
          }
          CHK[ci] = make_float2(sig ? -m1 : m1, m2);
        }
        team_sync(bar_id, G);
      }
      // ---- sweep-end test: a frame stops only when every check holds, so the checks of
      // the widest level are evaluated first (on the read-only flushed posterior); when one
      // fails, the full flush and syndrome are skipped (the same decision)
      bool full = t >= p.max_iter;
      if (!full && p.stop == CBP_STOP_SYNDROME) {
        bool fail = false;
        const int j1 = p.lvl_ptr[p.lvl_test + 1];
        for (int ci = p.lvl_ptr[p.lvl_test] + l; ci < j1; ci += G) {
          uint32_t par = 0;
          const int e1 = e0t[ci + 1];
          for (int e = e0t[ci]; e < e1; ++e) {
            const int v = static_cast<int>(lvl_rec<SHREC>(s_rec, led, e).vx & kSpMask);
            const float q = Q[v];
            const float2 pc = CHK[__ldg(p.last_chk + v)];
            const float b1 = fabsf(pc.x);
            const float rm = __fmul_rn(alpha, (fabsf(q) == b1) ? pc.y : b1);
            const float lb = __fadd_rn(q, (sign_bit(pc.x) ^ (q < 0.0f)) ? -rm : rm);
            par ^= lb < 0.0f ? 1u : 0u;
          }
          fail |= (par & 1u) != 0;
        }
        if (fail) s_unsat[g] = 1;
        team_sync(bar_id, G);
        full = *static_cast<volatile int*>(&s_unsat[g]) == 0;
        team_sync(bar_id, G);
        if (l == 0) s_unsat[g] = 0;
      }
      if (!full) continue;
      // ---- flushed posterior (Eq. s4e20 with the last check of v as c_j), decisions
      for (int vb = 0; vb < N; vb += G) {
        const int v = vb + l;
        bool neg = false;
        if (v < N) {
          const float q = Q[v];
          const float2 pc = CHK[__ldg(p.last_chk + v)];
          const float b1 = fabsf(pc.x);
          const float rm = __fmul_rn(alpha, (fabsf(q) == b1) ? pc.y : b1);
          const float lb = __fadd_rn(q, (sign_bit(pc.x) ^ (q < 0.0f)) ? -rm : rm);
          neg = lb < 0.0f;
          if (p.soft) p.soft[frame * N + v] = lb;
        }
        const unsigned wv = __ballot_sync(0xffffffffu, neg);
        if ((l & 31) == 0 && v < N) bits[v >> 5] = wv;
      }
      team_sync(bar_id, G);
      bool fail = false;
      for (int ci = l; ci < M; ci += G) {
        uint32_t par = 0;
        const int e1 = e0t[ci + 1];
        for (int e = e0t[ci]; e < e1; ++e) {
          const uint32_t v = lvl_rec<SHREC>(s_rec, led, e).vx & kSpMask;
          par ^= bits[v >> 5] >> (v & 31);
        }
        fail |= (par & 1u) != 0;
      }
      if (fail) s_unsat[g] = 1;
      team_sync(bar_id, G);
      const bool ok = *static_cast<volatile int*>(&s_unsat[g]) == 0;
      const bool done = (ok && p.stop == CBP_STOP_SYNDROME) || t >= p.max_iter;
      if (done) {
        uint32_t* ho = p.hard + frame * words;
        for (int w = l; w < words; w += G) ho[w] = bits[w];
        if (l == 0) p.iters[frame] = ok ? t : -t;
      }
      team_sync(bar_id, G);
      if (l == 0) s_unsat[g] = 0;
      team_sync(bar_id, G);
      if (done) break;
    }
  }
}

// Flooding sum-product BP (Sec. II-A, Eqs. s3e1, s3e2, s2e6, s2e7), the comparator, with the
// same lane groups: flooding has no order among checks, so the check phase takes the
// level-ordered checks on the lanes, then the variable phase the variables.  Per group,
// shared memory holds Lambda for every variable and the decision bits, the workspace the
// C2V messages by level-ordered edge; SHV instances also copy each edge's variable index,
// the check offsets and each variable's edges (ascending check index, the order of the
// posterior's sum) into shared memory.  The arithmetic is the lane-parallel flooding
// kernel's, operation for operation; a check's phi values stay in registers (D >= degree).
template <bool SHV, int D>
__global__ void __launch_bounds__(kLvlMaxThreads, 1) fbp_level_kernel(const KParams p) {
  extern __shared__ __align__(16) unsigned char smem[];
  const int G = p.lvl_lanes, F = p.F;
  const int N = p.N, M = p.M, E = p.E, words = p.words;
  const int tid = threadIdx.x;
  const int g = tid / G, l = tid - g * G;
  unsigned char* sp = smem;
  float4* s_tab = reinterpret_cast<float4*>(sp);
  sp += sizeof(float4) * kPhiSegments;
  int* s_unsat = reinterpret_cast<int*>(sp);
  sp += sizeof(int) * 16;
  uint32_t* s_v = reinterpret_cast<uint32_t*>(sp);
  int* s_e0 = reinterpret_cast<int*>(s_v + ((E + 3) & ~3));
  int* s_cp = s_e0 + ((M + 1 + 3) & ~3);
  int* s_ce = s_cp + ((N + 1 + 3) & ~3);
  if (SHV)
    sp += sizeof(int) * (2 * ((E + 3) & ~3) + ((M + 1 + 3) & ~3) + ((N + 1 + 3) & ~3));
  for (int i = tid; i < kPhiSegments; i += blockDim.x) s_tab[i] = p.phi_tab[i];
  if (tid < 16) s_unsat[tid] = 0;
  if (SHV) {
    for (int i = tid; i < E; i += blockDim.x) {
      s_v[i] = p.lvl_edge[i].x & kSpMask;
      s_ce[i] = p.lvl_cedge[i];
    }
    for (int i = tid; i <= M; i += blockDim.x) s_e0[i] = p.lvl_e0[i];
    for (int i = tid; i <= N; i += blockDim.x) s_cp[i] = p.lvl_cptr[i];
  }
  __syncthreads();
  if (g >= F) return;
  const int* e0t = SHV ? s_e0 : p.lvl_e0;
  const int* cpt = SHV ? s_cp : p.lvl_cptr;
  const int* cet = SHV ? s_ce : p.lvl_cedge;
  const LvlEdge* __restrict__ led = p.lvl_edge;
  float* lam = reinterpret_cast<float*>(sp) + static_cast<size_t>(g) * p.sh_frame;
  uint32_t* bits = reinterpret_cast<uint32_t*>(lam + ((N + 3) & ~3));
  const long long slot = static_cast<long long>(blockIdx.x) * F + g;
  float* R = p.ws + slot * p.ws_slot;
  const float4* tab = s_tab;
  const float xlo = p.phi_xlo;
  const int bar_id = 1 + g;
  auto var_of = [&](int e) -> int {
    return SHV ? static_cast<int>(s_v[e]) : static_cast<int>(__ldg(&led[e].x) & kSpMask);
  };

  for (long long frame = slot; frame < p.batch; frame += p.slots) {
    const float* L = p.llr + frame * N;
    bool bad = false;
    for (int v = l; v < N; v += G) {  // R = 0, so Lambda = L + 0 (Eq. s2e6)
      lam[v] = __fadd_rn(__ldg(L + v), 0.0f);
      bad |= non_finite(lam[v]);
    }
    if (bad) atomicOr(p.status, kStatusNonFiniteLlr);
    team_sync(bar_id, G);

    for (int t = 1;; ++t) {
      // ---- every check: Eqs. (s3e1), (s3e2)
      for (int ci = l; ci < M; ci += G) {
        const int k0 = e0t[ci], d = e0t[ci + 1] - k0;
        float ph[D];
        uint32_t neg = 0, sig = 0;
        float S = 0.0f;
#pragma unroll
        for (int j = 0; j < D; ++j) {
          if (j < d) {
            const float q = __fsub_rn(lam[var_of(k0 + j)], t > 1 ? R[k0 + j] : 0.0f);
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
            R[k0 + j] = (sig ^ ((neg >> j) & 1u)) ? -mag : mag;
          }
        }
      }
      team_sync(bar_id, G);
      // ---- posterior, Eq. (s2e6), in ascending check order; decisions, Eq. (s2e7)
      for (int vb = 0; vb < N; vb += G) {
        const int v = vb + l;
        bool ng = false;
        if (v < N) {
          float s = __ldg(L + v);
          const int c1 = cpt[v + 1];
          for (int k = cpt[v]; k < c1; ++k) s = __fadd_rn(s, R[cet[k]]);
          lam[v] = s;
          ng = s < 0.0f;
          if (p.soft) p.soft[frame * N + v] = s;
        }
        const unsigned wv = __ballot_sync(0xffffffffu, ng);
        if ((l & 31) == 0 && v < N) bits[v >> 5] = wv;
      }
      team_sync(bar_id, G);
      bool fail = false;
      for (int ci = l; ci < M; ci += G) {
        uint32_t par = 0;
        const int e1 = e0t[ci + 1];
        for (int e = e0t[ci]; e < e1; ++e) {
          const uint32_t v = static_cast<uint32_t>(var_of(e));
          par ^= bits[v >> 5] >> (v & 31);
        }
        fail |= (par & 1u) != 0;
      }
      if (fail) s_unsat[g] = 1;
      team_sync(bar_id, G);
      const bool ok = *static_cast<volatile int*>(&s_unsat[g]) == 0;
      const bool done = (ok && p.stop == CBP_STOP_SYNDROME) || t >= p.max_iter;
      if (done) {
        uint32_t* ho = p.hard + frame * words;
        for (int w = l; w < words; w += G) ho[w] = bits[w];
        if (l == 0) p.iters[frame] = ok ? t : -t;
      }
      team_sync(bar_id, G);
      if (l == 0) s_unsat[g] = 0;
      team_sync(bar_id, G);
      if (done) break;
    }
  }
}

}  // namespace

void* fbp_level_kernel_ptr(bool shv, int maxdeg) {
  if (maxdeg <= 8)
    return shv ? reinterpret_cast<void*>(&fbp_level_kernel<true, 8>)
               : reinterpret_cast<void*>(&fbp_level_kernel<false, 8>);
  if (maxdeg <= 16)
    return shv ? reinterpret_cast<void*>(&fbp_level_kernel<true, 16>)
               : reinterpret_cast<void*>(&fbp_level_kernel<false, 16>);
  return shv ? reinterpret_cast<void*>(&fbp_level_kernel<true, kMaxDeg>)
             : reinterpret_cast<void*>(&fbp_level_kernel<false, kMaxDeg>);
}

void* nms_level_kernel_ptr(bool shrec) {
  return shrec ? reinterpret_cast<void*>(&nms_level_kernel<true>)
               : reinterpret_cast<void*>(&nms_level_kernel<false>);
}

void* lbp_level_kernel_ptr(bool shv) {
  return shv ? reinterpret_cast<void*>(&lbp_level_kernel<true>)
             : reinterpret_cast<void*>(&lbp_level_kernel<false>);
}

void* level_kernel_ptr(bool shrec) {
  return shrec ? reinterpret_cast<void*>(&cbp_level_kernel<true>)
               : reinterpret_cast<void*>(&cbp_level_kernel<false>);
}

int level_max_threads() { return kLvlMaxThreads; }

}  // namespace cbp
