// Weighted CBP and its reverse-mode adjoint on sm_103a (the differentiable decoder).
//
// Forward (cbp_decode_weighted): T sweeps of CBP in log-tanh form, no stop, with the
// B2V message of Eq. (s4e18) scaled by w[tau][b]: tau is the sweep in which the
// predecessor check c_j formed its belief (this sweep if its base row comes earlier,
// else the previous sweep), b is c_j's base row; R^new = sgn * (w * phi(|S_cj - phi_v|)).
// The flushed posterior after sweep T (tau = T) is the output.  The state of every
// frame at the start of each segment of `ckpt` sweeps is saved in the workspace.
//
// Backward (cbp_decode_grad): from dLoss/dsoft, the adjoint of the flush, then for the
// segments in reverse: restore the segment's checkpoint, recompute its sweeps while
// recording per edge update (d = |S_cj| - phi_v, sgn * phi(|d|), Q^new), and run the
// sweeps backwards (base rows descending, a check's edges descending), propagating
// adjoints of Q*_v, phi(|Q*_v|), S_c and the C2V slots, and accumulating dLoss/dw.
// The adjoint of phi is the derivative of the evaluated cubic (phi_deriv).
// With one segment (ckpt = T) the forward records the tape of all T sweeps itself and
// keeps no checkpoint; the backward then recomputes nothing.  The adjoints of the
// check-beliefs live in shared memory when the CTA's frames' M floats each fit (GSS).
//
// Layout: F frames per CTA, Z lanes per frame (lane z owns check r*Z + z); all per-frame
// arrays live in the workspace, frame-major:
//   state   Q*[N] | phi[N] | S[M] (sign bit = sgn Omega) | R[E] ([base entry][lane])
//   adjoint gQ[N] | gP[N] | gS[M] | gR[E]
//   nseg checkpoints of the state (none when nseg = 1)
//   tape    d, sgn*mag, Q^new, each [ckpt][E]
#include "cbp_internal.cuh"

namespace cbp {
namespace {

__device__ __forceinline__ int mod_add(int a, int Z) { return a >= Z ? a - Z : a; }
__device__ __forceinline__ uint32_t sign_bit(float x) { return __float_as_uint(x) >> 31; }

struct Frame {
  float *Q, *P, *S, *R;       // state
  float *gQ, *gP, *gS, *gR;   // adjoint
  float* ck;                  // checkpoints
  float *td, *tm, *tq;        // tape
};

__device__ __forceinline__ Frame frame_view(const GParams& p, long long f) {
  Frame fr;
  float* b = p.ws + f * p.frame_floats;
  fr.Q = b;
  fr.P = b + p.N;
  fr.S = b + 2 * p.N;
  fr.R = b + 2 * p.N + p.M;
  float* a = b + p.st_floats;
  fr.gQ = a;
  fr.gP = a + p.N;
  fr.gS = a + 2 * p.N;
  fr.gR = a + 2 * p.N + p.M;
  fr.ck = b + 2 * p.st_floats;
  float* tp = fr.ck + static_cast<long long>(p.nseg > 1 ? p.nseg : 0) * p.st_floats;
  const long long te = static_cast<long long>(p.ckpt) * p.E;
  fr.td = tp;
  fr.tm = tp + te;
  fr.tq = tp + 2 * te;
  return fr;
}

struct Shared {
  float4* tab;
  BaseEdge* e;
  int* rptr;
  uint2* col;  // (last row | shift << 16)
  float* gw;   // [T*mb] weight gradients of this CTA
  float* w;    // [T*mb] the weights
  float* gs;   // [F][M] adjoints of the check-beliefs (backward with GSS)
};

__device__ Shared carve(unsigned char* smem, const GParams& p, bool load) {
  Shared sh;
  unsigned char* sp = smem;
  sh.tab = reinterpret_cast<float4*>(sp);
  sp += sizeof(float4) * kPhiSegments;
  sh.e = reinterpret_cast<BaseEdge*>(sp);
  sp += sizeof(BaseEdge) * p.nnzb;
  sh.rptr = reinterpret_cast<int*>(sp);
  sp += sizeof(int) * ((p.mb + 1 + 3) & ~3);
  sh.col = reinterpret_cast<uint2*>(sp);
  sp += sizeof(uint2) * ((p.nb + 1) & ~1);
  sh.gw = reinterpret_cast<float*>(sp);
  sp += sizeof(float) * p.T * p.mb;
  sh.w = reinterpret_cast<float*>(sp);
  sp += sizeof(float) * p.T * p.mb;
  sh.gs = reinterpret_cast<float*>(sp);
  if (load) {
    const int tid = threadIdx.x;
    for (int i = tid; i < kPhiSegments; i += blockDim.x) sh.tab[i] = p.phi_tab[i];
    for (int i = tid; i < p.nnzb; i += blockDim.x) sh.e[i] = p.edges[i];
    for (int i = tid; i <= p.mb; i += blockDim.x) sh.rptr[i] = p.rptr[i];
    for (int c = tid; c < p.nb; c += blockDim.x) {
      const ColEntry ce = p.cols[p.cptr[c + 1] - 1];
      sh.col[c] = make_uint2(uint32_t(ce.r) | (uint32_t(ce.s) << 16), 0u);
    }
    for (int i = tid; i < p.T * p.mb; i += blockDim.x) {
      sh.gw[i] = 0.0f;
      sh.w[i] = p.w[i];
    }
  }
  return sh;
}

// Copy a frame's state to / from a checkpoint (the Z lanes of the frame share the work).
__device__ __forceinline__ void copy_state(float* dst, const float* src, long long n, int z,
                                           int Z) {
  for (long long i = z; i < n; i += Z) dst[i] = src[i];
}

// Edges of a check handled together: their loads are issued before their updates.  The
// edges of one check touch distinct variables and distinct C2V slots (a predecessor slot
// lies in another base row), so the loads of a chunk never read what an earlier edge of
// the chunk writes; the updates keep the ascending (forward) or descending (adjoint) edge
// order, so every sum is formed in the same order as with one edge at a time.
constexpr int kGradChunk = 4;     // forward sweeps
constexpr int kGradChunkAdj = 3;  // adjoint sweeps (94 registers: 3 CTAs of 192 per SM)

// Forward sweeps t0..t1 (1-based, inclusive) of one frame, optionally recording the tape.
__device__ void forward_sweeps(const GParams& p, const Shared& sh, const Frame& fr, bool act,
                               int z, int t0, int t1, bool tape) {
  const int Z = p.Z;
  for (int t = t0; t <= t1; ++t) {
    const int ts = t - t0;
    for (int r = 0; r < p.mb; ++r) {
      if (act) {
        float Sacc = 0.0f;
        uint32_t sig = 0;
        const int k1 = sh.rptr[r + 1];
        for (int kb = sh.rptr[r]; kb < k1; kb += kGradChunk) {
          float q[kGradChunk], pv[kGradChunk], sj[kGradChunk], ro[kGradChunk];
          int vv[kGradChunk], zjj[kGradChunk];
#pragma unroll
          for (int j = 0; j < kGradChunk; ++j) {
            const int k = kb + j;
            if (k < k1) {
              const BaseEdge be = sh.e[k];
              const int zv = mod_add(z + be.s, Z);
              int zj = zv - be.ps;
              zj = zj < 0 ? zj + Z : zj;
              vv[j] = be.c * Z + zv;
              zjj[j] = zj;
              q[j] = fr.Q[vv[j]];
              pv[j] = fr.P[vv[j]];
              sj[j] = fr.S[be.pr * Z + zj];
              ro[j] = (!(be.flags & kSelf) && t > 1) ? fr.R[k * Z + z] : 0.0f;
            }
          }
#pragma unroll
          for (int j = 0; j < kGradChunk; ++j) {
            const int k = kb + j;
            if (k < k1) {
              const BaseEdge be = sh.e[k];
              const bool self = be.flags & kSelf;
              float Rn = 0.0f, d = 0.0f, smag = 0.0f;
              if (!(t == 1 && (be.flags & kFirst))) {
                d = __fsub_rn(fabsf(sj[j]), pv[j]);
                const float mag = phi_eval(fabsf(d), p.phi_xlo, sh.tab);
                const int tau = (be.pr < r) ? t : t - 1;
                const float wm = __fmul_rn(sh.w[(tau - 1) * p.mb + be.pr], mag);
                const bool neg = sign_bit(sj[j]) ^ (q[j] < 0.0f);
                Rn = neg ? -wm : wm;
                smag = neg ? -mag : mag;
                if (!self) fr.R[be.pe * Z + zjj[j]] = Rn;
              }
              const float rold = self ? Rn : ro[j];
              const float qn = __fsub_rn(__fadd_rn(q[j], Rn), rold);
              const float phn = phi_eval(fabsf(qn), p.phi_xlo, sh.tab);
              Sacc = __fadd_rn(Sacc, phn);
              sig ^= (qn < 0.0f);
              fr.Q[vv[j]] = qn;
              fr.P[vv[j]] = phn;
              if (tape) {
                const long long o = static_cast<long long>(ts) * p.E + k * Z + z;
                fr.td[o] = d;
                fr.tm[o] = smag;
                fr.tq[o] = qn;
              }
            }
          }
        }
        fr.S[r * Z + z] = sig ? -Sacc : Sacc;
      }
      __syncthreads();
    }
  }
}

// Warp-sum `x` and add it to sh.gw[idx] (every lane of the warp passes the same idx).
__device__ __forceinline__ void add_gw(const Shared& sh, int idx, float x) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) x += __shfl_down_sync(0xffffffffu, x, o);
  if ((threadIdx.x & 31) == 0 && x != 0.0f) atomicAdd(sh.gw + idx, x);
}

__global__ void __launch_bounds__(512) weighted_forward_kernel(const GParams p) {
  extern __shared__ __align__(16) unsigned char smem[];
  const Shared sh = carve(smem, p, true);
  const int Z = p.Z;
  const int f = threadIdx.x / Z, z = threadIdx.x - f * Z;
  const long long frame = static_cast<long long>(blockIdx.x) * p.F + f;
  const bool act = f < p.F && frame < p.batch;
  const Frame fr = frame_view(p, act ? frame : 0);
  __syncthreads();
  if (act) {
    const float* L = p.llr + frame * p.N;
    bool bad = false;
    for (int i = z; i < p.N; i += Z) {
      fr.Q[i] = L[i];  // Eq. (s4e15)
      bad |= non_finite(L[i]);
    }
    if (bad) atomicOr(p.status, kStatusNonFiniteLlr);
  }
  const bool one = p.nseg == 1;  // one segment: record the tape here, keep no checkpoint
  for (int s = 0; s < p.nseg; ++s) {
    const int t0 = s * p.ckpt + 1, t1 = min(p.T, (s + 1) * p.ckpt);
    __syncthreads();
    if (act && !one)
      copy_state(fr.ck + static_cast<long long>(s) * p.st_floats, fr.Q, p.st_floats, z, Z);
    __syncthreads();
    forward_sweeps(p, sh, fr, act, z, t0, t1, one);
  }
  if (act) {  // flushed posterior, tau = T
    for (int c = 0; c < p.nb; ++c) {
      const uint32_t l = sh.col[c].x;
      const int rk = int(l & 0xffff), sk = int(l >> 16);
      int zk = z - sk;
      zk = zk < 0 ? zk + Z : zk;
      const int v = c * Z + z;
      const float Sk = fr.S[rk * Z + zk];
      const float q = fr.Q[v];
      const float mag = phi_eval(fabsf(__fsub_rn(fabsf(Sk), fr.P[v])), p.phi_xlo, sh.tab);
      const float wm = __fmul_rn(sh.w[(p.T - 1) * p.mb + rk], mag);
      p.soft[frame * p.N + v] = __fadd_rn(q, (sign_bit(Sk) ^ (q < 0.0f)) ? -wm : wm);
    }
  }
}

template <bool GSS>
__global__ void __launch_bounds__(512) weighted_backward_kernel(const GParams p) {
  extern __shared__ __align__(16) unsigned char smem[];
  const Shared sh = carve(smem, p, true);
  const int Z = p.Z;
  const int f = threadIdx.x / Z, z = threadIdx.x - f * Z;
  const long long frame = static_cast<long long>(blockIdx.x) * p.F + f;
  const bool act = f < p.F && frame < p.batch;
  const Frame fr = frame_view(p, act ? frame : 0);
  const float xlo = p.phi_xlo;
  // adjoints of this frame's check-beliefs
  float* const gS = GSS ? sh.gs + static_cast<long long>(f < p.F ? f : 0) * p.M : fr.gS;
  if (act) {
    for (long long i = z; i < p.st_floats; i += Z) fr.gQ[i] = 0.0f;  // all adjoints
    if (GSS)
      for (int i = z; i < p.M; i += Z) gS[i] = 0.0f;
  }
  __syncthreads();
  // ---- adjoint of the flushed posterior (the state is the final one of the forward)
  for (int r = 0; r < p.mb; ++r) {
    for (int k = sh.rptr[r]; k < sh.rptr[r + 1]; ++k) {
      const BaseEdge be = sh.e[k];
      float gwx = 0.0f;
      if (act && (be.flags & kLast)) {
        const int v = be.c * Z + mod_add(z + be.s, Z);
        const int m = r * Z + z;
        const float Sm = fr.S[m], q = fr.Q[v];
        const float d = __fsub_rn(fabsf(Sm), fr.P[v]);
        const float mag = phi_eval(fabsf(d), xlo, sh.tab);
        const float sgn = (sign_bit(Sm) ^ (q < 0.0f)) ? -1.0f : 1.0f;
        const float w = sh.w[(p.T - 1) * p.mb + r];
        const float gl = p.gsoft[frame * p.N + v];
        fr.gQ[v] = gl;
        gwx = gl * sgn * mag;
        const float gd =
            gl * sgn * w * phi_deriv(fabsf(d), xlo, sh.tab) * (d < 0.0f ? -1.0f : 1.0f);
        gS[m] += gd;
        fr.gP[v] = -gd;
      }
      if (be.flags & kLast) add_gw(sh, (p.T - 1) * p.mb + r, gwx);
    }
  }
  __syncthreads();
  // ---- segments in reverse: recompute with the tape, then sweep backwards
  for (int s = p.nseg - 1; s >= 0; --s) {
    const int t0 = s * p.ckpt + 1, t1 = min(p.T, (s + 1) * p.ckpt);
    if (p.nseg > 1) {  // one segment: the forward recorded the tape
      if (act)
        copy_state(fr.Q, fr.ck + static_cast<long long>(s) * p.st_floats, p.st_floats, z, Z);
      __syncthreads();
      forward_sweeps(p, sh, fr, act, z, t0, t1, true);
    }
    for (int t = t1; t >= t0; --t) {
      const int ts = t - t0;
      for (int r = p.mb - 1; r >= 0; --r) {
        const int m = r * Z + z;
        float gSacc = 0.0f;
        if (act) {
          gSacc = gS[m];
          gS[m] = 0.0f;
        }
        const int k0 = sh.rptr[r];
        for (int kb = sh.rptr[r + 1] - 1; kb >= k0; kb -= kGradChunkAdj) {
          // loads of the chunk (edges kb, kb - 1, ...): the tape, the adjoints of the
          // variables and of the edge's own and predecessor C2V slots
          float td[kGradChunkAdj], tm[kGradChunkAdj], tq[kGradChunkAdj], gpv[kGradChunkAdj],
              gqv[kGradChunkAdj], gro[kGradChunkAdj], grs[kGradChunkAdj];
          int vv[kGradChunkAdj], zjj[kGradChunkAdj];
#pragma unroll
          for (int j = 0; j < kGradChunkAdj; ++j) {
            const int k = kb - j;
            if (act && k >= k0) {
              const BaseEdge be = sh.e[k];
              const int zv = mod_add(z + be.s, Z);
              int zj = zv - be.ps;
              zj = zj < 0 ? zj + Z : zj;
              vv[j] = be.c * Z + zv;
              zjj[j] = zj;
              const long long o = static_cast<long long>(ts) * p.E + k * Z + z;
              td[j] = fr.td[o];
              tm[j] = fr.tm[o];
              tq[j] = fr.tq[o];
              gpv[j] = fr.gP[vv[j]];
              gqv[j] = fr.gQ[vv[j]];
              gro[j] = fr.gR[k * Z + z];
              // a weight-1 edge is its own predecessor: its slot is read after the update
              grs[j] = (be.flags & kSelf) ? 0.0f : fr.gR[be.pe * Z + zj];
            }
          }
#pragma unroll
          for (int j = 0; j < kGradChunkAdj; ++j) {
            const int k = kb - j;
            if (k < k0) continue;  // uniform: the same edges for every lane
            const BaseEdge be = sh.e[k];
            const bool first = (t == 1) && (be.flags & kFirst);
            const int tau = (be.pr < r) ? t : t - 1;
            float gwx = 0.0f;
            if (act) {
              const int v = vv[j];
              const bool self = be.flags & kSelf;
              const float d = td[j], smag = tm[j], qn = tq[j];
              // phn = phi(|qn|) feeds phi_v and the sum S of this check
              const float gphn = gpv[j] + gSacc;
              const float gqn = gqv[j] + gphn * phi_deriv(fabsf(qn), xlo, sh.tab) *
                                             (qn < 0.0f ? -1.0f : 1.0f);
              const float gown = gro[j] - gqn;  // qn = (Q + Rn) - R[own]
              float gRn = gqn;                   // and Lambda = Q + Rn
              fr.gQ[v] = gqn;
              float gpn = 0.0f;
              if (first) {
                fr.gR[k * Z + z] = gown;
              } else {
                // R[slot] = Rn; the slot of a weight-1 edge is its own
                gRn += self ? gown : grs[j];
                if (self) {
                  fr.gR[k * Z + z] = 0.0f;
                } else {
                  fr.gR[k * Z + z] = gown;
                  fr.gR[be.pe * Z + zjj[j]] = 0.0f;
                }
                gwx = gRn * smag;  // Rn = sgn * w * mag
                const float w = sh.w[(tau - 1) * p.mb + be.pr];
                const float sgn = smag < 0.0f ? -1.0f : 1.0f;
                const float gd = gRn * sgn * w * phi_deriv(fabsf(d), xlo, sh.tab) *
                                 (d < 0.0f ? -1.0f : 1.0f);
                atomicAdd(gS + be.pr * Z + zjj[j], gd);  // d = |S_cj| - phi_v
                gpn = -gd;
              }
              fr.gP[v] = gpn;
            }
            if (!first) add_gw(sh, (tau - 1) * p.mb + be.pr, gwx);
          }
        }
        __syncthreads();
      }
    }
  }
  if (act && p.gllr)
    for (int i = z; i < p.N; i += Z) p.gllr[frame * p.N + i] = fr.gQ[i];  // Q* = L
  __syncthreads();
  for (int i = threadIdx.x; i < p.T * p.mb; i += blockDim.x)
    if (sh.gw[i] != 0.0f) atomicAdd(p.gw + i, sh.gw[i]);
}

}  // namespace

size_t grad_frame_floats(int N, int M, int E, int T, int ckpt) {
  const size_t st = (2 * static_cast<size_t>(N) + M + E + 3) & ~static_cast<size_t>(3);
  const size_t nseg = (T + ckpt - 1) / ckpt;
  const size_t f = 2 * st + (nseg > 1 ? nseg * st : 0) + 3 * static_cast<size_t>(ckpt) * E;
  return (f + 63) & ~static_cast<size_t>(63);
}

cudaError_t grad_set_smem(int bytes) {
  cudaError_t e = cudaFuncSetAttribute(weighted_forward_kernel,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
  if (e != cudaSuccess) return e;
  e = cudaFuncSetAttribute(weighted_backward_kernel<true>,
                           cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
  if (e != cudaSuccess) return e;
  return cudaFuncSetAttribute(weighted_backward_kernel<false>,
                              cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
}

cudaError_t launch_weighted_forward(const GParams& p, int grid, int threads, size_t smem,
                                    cudaStream_t st) {
  weighted_forward_kernel<<<grid, threads, smem, st>>>(p);
  return cudaGetLastError();
}

cudaError_t launch_weighted_backward(const GParams& p, int grid, int threads, size_t smem,
                                     cudaStream_t st) {
  if (p.gs_shared)
    weighted_backward_kernel<true><<<grid, threads, smem + p.gs_bytes, st>>>(p);
  else
    weighted_backward_kernel<false><<<grid, threads, smem, st>>>(p);
  return cudaGetLastError();
}

}  // namespace cbp
