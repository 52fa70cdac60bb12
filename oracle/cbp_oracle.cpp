// CPU oracle for check-belief propagation (CBP) decoding and its comparators.
//
// TEST INFRASTRUCTURE ONLY.  Only tests/, __graft_entry__.smoke() and bench.py's
// CPU-baseline leg may load this library.  It shares no code, header, table or
// constant generator with the CUDA path; the two meet only in the seeded inputs.
//
// Everything here is plain, sequential and unoptimised on purpose: one frame at a
// time, the expanded Tanner graph held as index lists, every message update
// written in the paper's notation and order.
//
//   phi(x) = -log tanh(x/2)                                    Eq. (s2e5)
//   CBP, log-tanh form: Step 1 (Eqs. s4e15-s4e17), Step 2 a)-e) (Eqs. s4e18-s4e23),
//     with the check-belief kept as S_c = sum phi(|Q|) and its sign (Appendix A,
//     Eqs. ae2-ae5); a literal Omega-domain version (Eqs. s4e5, s4e6, s4e12, s4e13)
//     runs in FP64 beside it.
//   CBP normalized min-sum: Eqs. (s4e18xx), (s4e21xx), Sec. IV-D.
//   Layered BP (LBP): Eqs. (s2e10), (s2e12) with the shared-value check update (s3e2).
//   Flooding BP (FBP): Eqs. (s2e3)/(s3e1), (s2e4)/(s3e2), (s2e6), (s2e7).
//   Weighted CBP (learnable scale per sweep x base row on the B2V message) and its
//   reverse-mode adjoint in FP64, for the differentiable decoder.
//
// Readings of the paper (where it is silent or garbled):
//   * Eq. (s4e22) stores R_{c_i->v} <- R^new_{c_j->v}; read as R_{c_j->v} <- R^new_{c_j->v}
//     (the new C2V of the predecessor check), which makes CBP layered BP with each
//     C2V computed at the variable's next visit.
//   * A variable with no earlier visit has no C2V to add: R^new = 0 (instead of the
//     psi^-(infinity, Q) of "initialize the first check-node as the latest updated one").
//   * A check of degree 1 in its column (c_j == c_i): R[c_j,v] is written before
//     R[c_i,v] is read, so Q^new = (Q + R^new) - R^new.
//   * Fold and V2C order: variables of a check in ascending index; Lambda = Q + R^new
//     is rounded before Q^new = Lambda - R_old.  No fused multiply-add contraction.
//   * sgn(x) is negative iff x < 0, so +0 and -0 count as positive; x_hat = [Lambda < 0].
//   * Stop: the syndrome H x_hat^T = 0 (suppressed text of Sec. II-A) tested after every
//     full sweep on the flushed posterior Lambda_bar_v = Q_v + B2V(last check of v, v),
//     a read-only evaluation of Eq. (s4e20) at the end of the sweep.  iters = sweeps run,
//     negated when the syndrome is still non-zero after max_iter sweeps.
//   * Paper-literal stop (CBP log-tanh only): Eq. (s4e24) read as a window of M
//     consecutive check updates (the check-beliefs number M, not N), counted across
//     sweep boundaries, each leaving Omega > 0 (Eq. s4e2) and no flip of a posterior
//     sign of Eq. (s4e20) against that variable's previous posterior (initially the
//     channel LLR).  Decoding stops right after the M-th such update, possibly in the
//     middle of a sweep; the output is the sign of each variable's latest Lambda^new
//     (Step 3, "generated in the V2C phase").
//   * CBP min-sum: minima of |Q| kept unscaled; strict '<' so the first of equal values
//     wins; B2V picks min2 when |Q*_v| equals min1; R = alpha * min with sign.
//   * phi in FP32: phi(clamp(x, X_LO, X_HI)), X_HI = 30, X_LO = fl32(phi(30)),
//     evaluated as a cubic Taylor polynomial around the nearest centre of a fixed
//     grid (32 per binade below 2, step 1/16 from 2 to 30) with coefficients taken
//     from the closed-form derivatives of phi in FP64 and rounded to FP32.
//     In FP64: phi(clamp(x, phi(50), 50)) from libm.
#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <limits>
#include <thread>
#include <vector>

namespace {

// ---------------------------------------------------------------------------
// phi, Eq. (s2e5)
// ---------------------------------------------------------------------------
constexpr float kXhi32 = 30.0f;
constexpr float kXlo32 = 0x1.a56e0cp-43f;  // fl32(phi(30)); pinned by a test
constexpr double kXhi64 = 50.0;

double phi_libm(double x) { return std::log1p(2.0 / std::expm1(x)); }

double xlo64() {
  static const double v = phi_libm(kXhi64);
  return v;
}

double phi64(double x) {
  if (!(x > xlo64())) x = xlo64();  // also maps NaN to the lower clamp
  if (x > kXhi64) x = kXhi64;
  return phi_libm(x);
}

inline uint32_t f2u(float f) { uint32_t u; std::memcpy(&u, &f, 4); return u; }
inline float u2f(uint32_t u) { float f; std::memcpy(&f, &u, 4); return f; }

// Grid of expansion centres.  Below 2: the FP32 values whose low 18 mantissa bits
// are zero (32 centres per binade), from 2^-43 (bit pattern 2688 << 18) to 2.0.
// From 2 to 30: k/16 for k = 32..480.
constexpr int kLogBase = 2688;       // (bits of 2^-43) >> 18
constexpr int kLogCount = 1409;      // centres 2^-43 ... 2.0
constexpr int kUniCount = 449;       // centres 2.0, 2.0625, ..., 30.0
constexpr int kSegments = kLogCount + kUniCount;

struct PhiTable {
  std::vector<float> c;  // 4 coefficients per centre: value, then scaled derivatives
  PhiTable() : c(4 * kSegments) {
    for (int i = 0; i < kSegments; ++i) {
      double m, h;
      if (i < kLogCount) {
        uint32_t cb = static_cast<uint32_t>(kLogBase + i) << 18;
        m = static_cast<double>(u2f(cb));
        int e = static_cast<int>((cb >> 23) & 0xffu) - 127;
        h = std::ldexp(1.0, e);           // t = (x - m) / 2^e
      } else {
        m = (32 + (i - kLogCount)) / 16.0;
        h = 1.0 / 16.0;                   // t = (x - m) * 16
      }
      // phi(m), phi'(m) = -1/sinh m, phi''(m) = cosh m / sinh^2 m,
      // phi'''(m) = -(cosh^2 m + 1) / sinh^3 m; Taylor coefficients times h^k.
      double sh = std::sinh(m), ch = std::cosh(m);
      double r = h / sh;
      double d0 = phi_libm(m);
      double d1 = -r;
      double d2 = 0.5 * ch * (r * r);
      double d3 = -(ch * ch + 1.0) * (r * r * r) / 6.0;
      c[4 * i + 0] = static_cast<float>(d0);
      c[4 * i + 1] = static_cast<float>(d1);
      c[4 * i + 2] = static_cast<float>(d2);
      c[4 * i + 3] = static_cast<float>(d3);
    }
  }
};

const PhiTable& phi_table() {
  static const PhiTable t;
  return t;
}

float phi32(float x) {
  x = std::fmin(std::fmax(x, kXlo32), kXhi32);  // fmax drops a NaN operand
  int i;
  float t;
  if (x < 2.0f) {
    uint32_t cb = (f2u(x) + 0x20000u) & 0xFFFC0000u;  // nearest centre
    i = static_cast<int>(cb >> 18) - kLogBase;
    float m = u2f(cb);
    float inv = u2f((254u - (cb >> 23)) << 23);       // 2^-e of the centre
    t = (x - m) * inv;
  } else {
    float u = x * 16.0f;
    float k = std::rint(u);
    t = u - k;
    i = static_cast<int>(k) - 32 + kLogCount;
  }
  const float* c = &phi_table().c[4 * i];
  float p = std::fma(c[3], t, c[2]);
  p = std::fma(p, t, c[1]);
  p = std::fma(p, t, c[0]);
  return p;
}

inline float phi_t(float x) { return phi32(x); }
inline double phi_t(double x) { return phi64(x); }

// ---------------------------------------------------------------------------
// Tanner graph of a QC code:  H[r*Z+i, c*Z+(i+s)%Z] = 1
// ---------------------------------------------------------------------------
struct Graph {
  int N = 0, M = 0, E = 0, Z = 1, mb = 0;
  std::vector<int> cptr, cvar, echk;  // check -> edges (ascending variable); edge -> check
  std::vector<int> vptr, vedge;       // variable -> edges (ascending check)
};

enum { CBP_SP = 0, CBP_NMS = 1, LBP_NMS = 2, FBP_SP = 3, LBP_SP = 4, CBP_SP_OMEGA = 5 };

// counters, per decode call (summed over frames)
enum { C_SWEEPS = 0, C_B2V, C_V2C, C_C2B, C_SUMS, C_PRODUCTS, C_C2V, C_FLUSH, C_COUNT };

constexpr float kFlagEps = 1e-4f;

template <class T>
inline T sgn_apply(bool neg, T mag) { return neg ? -mag : mag; }

template <class T>
struct Frame {
  const Graph& g;
  const T* L;
  int max_iter, stop;
  T alpha;
  uint8_t* hard;
  T* soft;
  int32_t iters = 0;
  uint8_t flag = 0;
  int64_t* cnt;
  // work arrays
  std::vector<T> Q, Ph, S, S2, R, Lam, Lb;
  std::vector<uint8_t> sg;
  std::vector<int> last;
  Frame(const Graph& g_, int64_t* cnt_) : g(g_), cnt(cnt_) {}

  void note_small(T v) {
    if (std::fabs(v) < static_cast<T>(kFlagEps)) flag |= 1;
  }

  // H x_hat^T == 0 ?
  bool syndrome_zero() const {
    for (int m = 0; m < g.M; ++m) {
      int p = 0;
      for (int e = g.cptr[m]; e < g.cptr[m + 1]; ++e) p ^= hard[g.cvar[e]];
      if (p) return false;
    }
    return true;
  }

  void finish_sweep(int t, bool& done) {
    cnt[C_SWEEPS] += 1;
    bool ok = syndrome_zero();
    if (ok && stop == 0) {
      iters = t;
      done = true;
    } else if (t == max_iter) {
      iters = ok ? t : -t;
      done = true;
    }
  }

  // ---- CBP, log-tanh form, S-domain (Step 1-3 of Sec. IV-C) ----
  void cbp_sp() {
    const int N = g.N, M = g.M, E = g.E;
    Q.assign(L, L + N);                // Eq. (s4e15): Q_{v->c*} = L_v
    Ph.assign(N, T(0));                // phi(|Q_{v->c*}|) of the latest V2C
    S.assign(M, T(0));                 // Eq. (s4e16): Omega = inf  <=>  S = 0
    sg.assign(M, 0);
    R.assign(E, T(0));                 // Eq. (s4e17)
    last.assign(N, -1);                // edge of the latest updated check of v
    // Paper-literal stop (stop == 2), Step 2 (3) and Step 3 of Sec. IV-C: the decoding
    // succeeds once M consecutive check updates each leave Omega > 0 (Eq. s4e2) and flip
    // no posterior sign of Eq. (s4e20) (Eq. s4e24); the output is the hard decision of
    // the latest V2C phase.  pneg[v] = [latest Lambda^new_v < 0], initially [L_v < 0].
    const bool window = stop == 2;
    std::vector<uint8_t> pneg;
    long long win = 0;
    if (window) {
      pneg.resize(N);
      for (int v = 0; v < N; ++v) pneg[v] = L[v] < T(0);
      Lam.assign(L, L + N);
    }
    bool done = false;
    for (int t = 1; t <= max_iter && !done; ++t) {
      for (int m = 0; m < M && !done; ++m) {  // sequential order of check-nodes
        T Sacc = T(0);
        int sig = 0;
        bool flip = false;
        for (int e = g.cptr[m]; e < g.cptr[m + 1]; ++e) {
          const int v = g.cvar[e];
          T Rn = T(0);
          const int le = last[v];
          if (le >= 0) {               // a) c_j = latest updated check of v
            const int cj = g.echk[le];
            // b) B2V, Eq. (s4e18) via Eq. (s4e13): exclude phi(|Q|) from S_{c_j}
            T mag = phi_t(std::fabs(S[cj] - Ph[v]));
            Rn = sgn_apply(static_cast<bool>(sg[cj] ^ (Q[v] < T(0))), mag);
            R[le] = Rn;                // e) store R_{c_j->v}
            cnt[C_PRODUCTS] += 1;
          }
          cnt[C_B2V] += 1;
          // c) V2C, Eqs. (s4e20), (s4e19)
          T lam = Q[v] + Rn;
          T qn = lam - R[e];
          cnt[C_V2C] += 1;
          cnt[C_SUMS] += 2;
          if (window) {                // Eq. (s4e24): sign flip of the posterior?
            const uint8_t neg = lam < T(0);
            flip |= neg != pneg[v];
            pneg[v] = neg;
            Lam[v] = lam;
          }
          // d) C2B, Eq. (s4e21) in the S-domain
          T ph = phi_t(std::fabs(qn));
          Sacc = Sacc + ph;
          sig ^= (qn < T(0));
          cnt[C_C2B] += 1;
          cnt[C_PRODUCTS] += 1;
          note_small(qn);
          Q[v] = qn;                   // e) Q_{v->c*} <- Q^new
          Ph[v] = ph;
          last[v] = e;
        }
        S[m] = Sacc;                   // Eq. (s4e23)
        sg[m] = static_cast<uint8_t>(sig);
        if (window) {
          win = (sig == 0 && !flip) ? win + 1 : 0;
          if (win >= M) {              // success, Step 3: x_hat of the latest V2C phase
            for (int v = 0; v < N; ++v) hard[v] = pneg[v];
            if (soft) std::copy(Lam.begin(), Lam.end(), soft);
            cnt[C_SWEEPS] += 1;
            iters = t;
            done = true;
          }
        }
      }
      if (window) {
        if (!done && t == max_iter) {
          for (int v = 0; v < N; ++v) hard[v] = pneg[v];
          if (soft) std::copy(Lam.begin(), Lam.end(), soft);
          cnt[C_SWEEPS] += 1;
          iters = -t;
          done = true;
        } else if (!done) {
          cnt[C_SWEEPS] += 1;
        }
        continue;
      }
      // flushed posterior and hard decision, Eqs. (s4e20), (s2e7)
      for (int v = 0; v < N; ++v) {
        const int cj = g.echk[last[v]];
        T mag = phi_t(std::fabs(S[cj] - Ph[v]));
        T lb = Q[v] + sgn_apply(static_cast<bool>(sg[cj] ^ (Q[v] < T(0))), mag);
        cnt[C_FLUSH] += 1;
        note_small(lb);
        hard[v] = lb < T(0);
        if (soft) soft[v] = lb;
      }
      finish_sweep(t, done);
    }
  }

  // ---- CBP in the literal Omega domain, Eqs. (s4e5)/(s4e6), (s4e12)/(s4e13) ----
  static T sgn(T x) { return x < T(0) ? T(-1) : T(1); }
  static T psi_plus(T x, T y) {
    return sgn(x) * sgn(y) * phi_t(phi_t(std::fabs(x)) + phi_t(std::fabs(y)));
  }
  static T psi_minus(T x, T y) {
    return sgn(x) * sgn(y) * phi_t(std::fabs(phi_t(std::fabs(x)) - phi_t(std::fabs(y))));
  }
  void cbp_sp_omega() {
    const int N = g.N, M = g.M, E = g.E;
    Q.assign(L, L + N);
    S.assign(M, std::numeric_limits<T>::infinity());  // Omega_c = inf, Eq. (s4e16)
    R.assign(E, T(0));
    last.assign(N, -1);
    bool done = false;
    for (int t = 1; t <= max_iter && !done; ++t) {
      for (int m = 0; m < M; ++m) {
        T Om = std::numeric_limits<T>::infinity();  // Omega^(-1) = inf
        for (int e = g.cptr[m]; e < g.cptr[m + 1]; ++e) {
          const int v = g.cvar[e];
          T Rn = T(0);
          if (last[v] >= 0) {
            Rn = psi_minus(S[g.echk[last[v]]], Q[v]);  // Eq. (s4e18)
            R[last[v]] = Rn;
          }
          T qn = (Q[v] + Rn) - R[e];                  // Eq. (s4e19)
          Om = psi_plus(Om, qn);                      // Eq. (s4e21)
          Q[v] = qn;
          last[v] = e;
        }
        S[m] = Om;                                    // Eq. (s4e23)
      }
      for (int v = 0; v < N; ++v) {
        T lb = Q[v] + psi_minus(S[g.echk[last[v]]], Q[v]);
        hard[v] = lb < T(0);
        if (soft) soft[v] = lb;
      }
      finish_sweep(t, done);
    }
  }

  // ---- CBP normalized min-sum, Eqs. (s4e18xx), (s4e21xx) ----
  void cbp_nms() {
    const int N = g.N, M = g.M, E = g.E;
    const T inf = std::numeric_limits<T>::infinity();
    Q.assign(L, L + N);
    S.assign(M, inf);    // min1 of |Q| per check (unscaled)
    S2.assign(M, inf);   // min2
    sg.assign(M, 0);
    R.assign(E, T(0));
    last.assign(N, -1);
    bool done = false;
    auto b2v = [&](int cj, T q) {
      T a = std::fabs(q);
      T mag = (a == S[cj]) ? S2[cj] : S[cj];
      return sgn_apply(static_cast<bool>(sg[cj] ^ (q < T(0))), alpha * mag);
    };
    for (int t = 1; t <= max_iter && !done; ++t) {
      for (int m = 0; m < M; ++m) {
        T m1 = inf, m2 = inf;
        int sig = 0;
        for (int e = g.cptr[m]; e < g.cptr[m + 1]; ++e) {
          const int v = g.cvar[e];
          T Rn = T(0);
          if (last[v] >= 0) {
            Rn = b2v(g.echk[last[v]], Q[v]);
            R[last[v]] = Rn;
            cnt[C_PRODUCTS] += 1;
          }
          cnt[C_B2V] += 1;
          T lam = Q[v] + Rn;
          T qn = lam - R[e];
          cnt[C_V2C] += 1;
          cnt[C_SUMS] += 2;
          T a = std::fabs(qn);
          if (a == m1 || a == m2) flag |= 2;
          if (a < m1) {
            m2 = m1;
            m1 = a;
          } else if (a < m2) {
            m2 = a;
          }
          sig ^= (qn < T(0));
          cnt[C_C2B] += 1;
          cnt[C_PRODUCTS] += 1;
          note_small(qn);
          Q[v] = qn;
          last[v] = e;
        }
        S[m] = m1;
        S2[m] = m2;
        sg[m] = static_cast<uint8_t>(sig);
      }
      for (int v = 0; v < N; ++v) {
        T lb = Q[v] + b2v(g.echk[last[v]], Q[v]);
        cnt[C_FLUSH] += 1;
        note_small(lb);
        hard[v] = lb < T(0);
        if (soft) soft[v] = lb;
      }
      finish_sweep(t, done);
    }
  }

  // ---- layered BP, Eqs. (s2e10), (s2e12); check update in the form of Eq. (s3e2) ----
  void lbp(bool minsum) {
    const int N = g.N, M = g.M, E = g.E;
    const T inf = std::numeric_limits<T>::infinity();
    Lam.assign(L, L + N);
    R.assign(E, T(0));
    std::vector<T> q, p;
    bool done = false;
    for (int t = 1; t <= max_iter && !done; ++t) {
      for (int m = 0; m < M; ++m) {
        const int b = g.cptr[m], d = g.cptr[m + 1] - b;
        q.resize(d);
        p.resize(d);
        int sig = 0;
        T Sacc = T(0), m1 = inf, m2 = inf;
        int idx = -1;
        for (int k = 0; k < d; ++k) {           // Eq. (s2e10)
          const int v = g.cvar[b + k];
          q[k] = Lam[v] - R[b + k];
          cnt[C_V2C] += 1;
          cnt[C_SUMS] += 1;
          note_small(q[k]);
          sig ^= (q[k] < T(0));
          if (minsum) {
            T a = std::fabs(q[k]);
            if (a == m1 || a == m2) flag |= 2;
            if (a < m1) {
              m2 = m1;
              m1 = a;
              idx = k;
            } else if (a < m2) {
              m2 = a;
            }
          } else {
            p[k] = phi_t(std::fabs(q[k]));
            Sacc = Sacc + p[k];                  // shared sum of Eq. (s3e2)
            cnt[C_PRODUCTS] += 1;
          }
        }
        for (int k = 0; k < d; ++k) {           // Eq. (s3e2), then Eq. (s2e12)
          const int v = g.cvar[b + k];
          T mag = minsum ? alpha * (k == idx ? m2 : m1) : phi_t(std::fabs(Sacc - p[k]));
          T Rn = sgn_apply(static_cast<bool>(sig ^ (q[k] < T(0))), mag);
          R[b + k] = Rn;
          Lam[v] = q[k] + Rn;
          cnt[C_C2V] += 1;
          cnt[C_SUMS] += 1;
          if (!minsum) cnt[C_PRODUCTS] += 1;
        }
      }
      for (int v = 0; v < N; ++v) {
        note_small(Lam[v]);
        hard[v] = Lam[v] < T(0);
        if (soft) soft[v] = Lam[v];
      }
      finish_sweep(t, done);
    }
  }

  // ---- flooding BP: Eqs. (s3e1), (s3e2), (s2e6), (s2e7) ----
  void fbp() {
    const int N = g.N, M = g.M, E = g.E;
    R.assign(E, T(0));
    Lam.assign(N, T(0));
    auto posterior = [&]() {                   // Eq. (s2e6), ascending check order
      for (int v = 0; v < N; ++v) {
        T s = L[v];
        for (int k = g.vptr[v]; k < g.vptr[v + 1]; ++k) s = s + R[g.vedge[k]];
        Lam[v] = s;
      }
    };
    posterior();
    std::vector<T> q, p;
    bool done = false;
    for (int t = 1; t <= max_iter && !done; ++t) {
      for (int m = 0; m < M; ++m) {
        const int b = g.cptr[m], d = g.cptr[m + 1] - b;
        q.resize(d);
        p.resize(d);
        int sig = 0;
        T Sacc = T(0);
        for (int k = 0; k < d; ++k) {
          q[k] = Lam[g.cvar[b + k]] - R[b + k];  // Eq. (s3e1): total minus own
          cnt[C_V2C] += 1;
          note_small(q[k]);
          sig ^= (q[k] < T(0));
          p[k] = phi_t(std::fabs(q[k]));
          Sacc = Sacc + p[k];
        }
        for (int k = 0; k < d; ++k) {            // Eq. (s3e2)
          R[b + k] = sgn_apply(static_cast<bool>(sig ^ (q[k] < T(0))),
                               phi_t(std::fabs(Sacc - p[k])));
          cnt[C_C2V] += 1;
        }
      }
      posterior();
      for (int v = 0; v < N; ++v) {
        note_small(Lam[v]);
        hard[v] = Lam[v] < T(0);
        if (soft) soft[v] = Lam[v];
      }
      finish_sweep(t, done);
    }
  }
};

// ---------------------------------------------------------------------------
// Weighted CBP (a learnable scale per sweep x base row on the B2V message) and its
// reverse-mode adjoint.  Reading: the C2V message R^new_{c_j->v} of Eq. (s4e18) is
// multiplied by w[tau][b] where tau is the sweep in which Omega_{c_j} was formed and b
// the base row of c_j; the flushed posterior after the last sweep uses tau = T.
// T sweeps, no early stop.  w = 1 gives CBP (log-tanh form).  Rn = sgn * (w * mag).
// ---------------------------------------------------------------------------
template <class T>
struct WStep {             // one edge update of the forward, for the reverse pass
  int v, e, ej, cj, ci, widx;  // ej = -1: first visit (no B2V)
  T d, mag, sgn, w, qn, phn;
};

template <class T>
inline T dphi_t(T x);  // derivative of phi (0 outside the clamp range)
template <>
inline double dphi_t<double>(double x) {
  if (!(x > xlo64()) || x > kXhi64) return 0.0;
  return -1.0 / std::sinh(x);
}

template <class T>
void weighted_forward(const Graph& g, const T* L, const T* w, int Tsw, T* soft,
                      std::vector<WStep<T>>* tape, std::vector<T>* lb_parts) {
  const int N = g.N, M = g.M, E = g.E;
  std::vector<T> Q(L, L + N), Ph(N, T(0)), S(M, T(0)), R(E, T(0));
  std::vector<uint8_t> sg(M, 0);
  std::vector<int> last(N, -1), formed(M, 0);
  for (int t = 1; t <= Tsw; ++t)
    for (int m = 0; m < M; ++m) {
      T Sacc = T(0);
      int sig = 0;
      for (int e = g.cptr[m]; e < g.cptr[m + 1]; ++e) {
        const int v = g.cvar[e];
        WStep<T> st{};
        st.v = v;
        st.e = e;
        st.ci = m;
        st.ej = last[v];
        T Rn = T(0);
        if (last[v] >= 0) {
          const int cj = g.echk[last[v]];
          st.cj = cj;
          st.d = S[cj] - Ph[v];
          st.mag = phi_t(std::fabs(st.d));
          st.sgn = (sg[cj] ^ (Q[v] < T(0))) ? T(-1) : T(1);
          st.widx = (formed[cj] - 1) * g.mb + cj / g.Z;
          st.w = w[st.widx];
          Rn = st.sgn * (st.w * st.mag);
          R[last[v]] = Rn;
        }
        const T lam = Q[v] + Rn;
        const T qn = lam - R[e];
        const T ph = phi_t(std::fabs(qn));
        Sacc = Sacc + ph;
        sig ^= (qn < T(0));
        st.qn = qn;
        st.phn = ph;
        Q[v] = qn;
        Ph[v] = ph;
        last[v] = e;
        if (tape) tape->push_back(st);
      }
      S[m] = Sacc;
      sg[m] = static_cast<uint8_t>(sig);
      formed[m] = t;
    }
  // flushed posterior with tau = T
  if (lb_parts) lb_parts->assign(4 * static_cast<size_t>(N), T(0));
  for (int v = 0; v < N; ++v) {
    const int cj = g.echk[last[v]];
    const T d = S[cj] - Ph[v];
    const T mag = phi_t(std::fabs(d));
    const T sgn = (sg[cj] ^ (Q[v] < T(0))) ? T(-1) : T(1);
    const int widx = (Tsw - 1) * g.mb + cj / g.Z;
    soft[v] = Q[v] + sgn * (w[widx] * mag);
    if (lb_parts) {
      (*lb_parts)[4 * v + 0] = d;
      (*lb_parts)[4 * v + 1] = mag;
      (*lb_parts)[4 * v + 2] = sgn;
      (*lb_parts)[4 * v + 3] = static_cast<T>(widx);
    }
  }
}

// dLoss/dw (accumulated into gw) and dLoss/dL (into gL) from gsoft = dLoss/dLambda_bar.
void weighted_backward(const Graph& g, const double* L, const double* w, int Tsw,
                       const double* gsoft, double* gw, double* gL) {
  const int N = g.N, M = g.M, E = g.E;
  std::vector<WStep<double>> tape;
  std::vector<double> soft(N), parts;
  weighted_forward<double>(g, L, w, Tsw, soft.data(), &tape, &parts);
  std::vector<double> gQ(N, 0.0), gP(N, 0.0), gS(M, 0.0), gR(E, 0.0);
  std::vector<int> last(N, -1);
  // final state: the last check of every variable is the check of its last edge step
  for (const auto& st : tape) last[st.v] = st.ci;
  for (int v = 0; v < N; ++v) {  // flushed posterior, reversed
    const double d = parts[4 * v], mag = parts[4 * v + 1], sgn = parts[4 * v + 2];
    const int widx = static_cast<int>(parts[4 * v + 3]);
    const double gl = gsoft[v];
    gQ[v] += gl;
    gw[widx] += gl * sgn * mag;
    const double gd = gl * sgn * w[widx] * dphi_t<double>(std::fabs(d)) * (d < 0 ? -1.0 : 1.0);
    gS[last[v]] += gd;
    gP[v] -= gd;
  }
  // edge updates in reverse order; the adjoint of a check's S starts at its last use
  double gSacc = 0.0;
  int cur = -1;
  for (size_t k = tape.size(); k-- > 0;) {
    const WStep<double>& st = tape[k];
    if (st.ci != cur) {   // reverse of S[ci] = sum of phi(|Q^new|) over the check
      cur = st.ci;
      gSacc = gS[cur];
      gS[cur] = 0.0;
    }
    const int v = st.v;
    const double gphn = gP[v] + gSacc;                          // phn = phi(|qn|)
    const double gqn = gQ[v] + gphn * dphi_t<double>(std::fabs(st.qn)) * (st.qn < 0 ? -1.0 : 1.0);
    const double glam = gqn;                                    // qn = lam - R[e]
    gR[st.e] -= gqn;                                            // R[e] read
    double gRn = glam;                                          // lam = Q + Rn
    gQ[v] = glam;                                               // adjoint of the old Q*_v
    gP[v] = 0.0;
    if (st.ej >= 0) {
      gRn += gR[st.ej];                                         // R[ej] = Rn (write)
      gR[st.ej] = 0.0;
      gw[st.widx] += gRn * st.sgn * st.mag;                     // Rn = sgn * w * mag
      const double gd = gRn * st.sgn * st.w * dphi_t<double>(std::fabs(st.d)) *
                        (st.d < 0 ? -1.0 : 1.0);
      gS[st.cj] += gd;                                          // d = S[cj] - Ph[v]
      gP[v] = -gd;
    }
  }
  for (int v = 0; v < N; ++v) gL[v] += gQ[v];
}

bool build_graph(const int32_t* base, int mb, int nb, int Z, Graph& g) {
  if (!base || mb < 1 || nb < 1 || Z < 1) return false;
  for (int i = 0; i < mb * nb; ++i)
    if (base[i] < -1 || base[i] >= Z) return false;
  for (int r = 0; r < mb; ++r) {
    int d = 0;
    for (int c = 0; c < nb; ++c) d += base[r * nb + c] >= 0;
    if (d < 2) return false;           // a degree-1 check pins its variable: rejected
  }
  for (int c = 0; c < nb; ++c) {
    int w = 0;
    for (int r = 0; r < mb; ++r) w += base[r * nb + c] >= 0;
    if (w < 1) return false;           // a variable in no check: rejected
  }
  g.N = nb * Z;
  g.M = mb * Z;
  g.Z = Z;
  g.mb = mb;
  g.cptr.assign(1, 0);
  g.cvar.clear();
  g.echk.clear();
  for (int r = 0; r < mb; ++r)
    for (int i = 0; i < Z; ++i) {
      for (int c = 0; c < nb; ++c) {
        int s = base[r * nb + c];
        if (s < 0) continue;
        g.cvar.push_back(c * Z + (i + s) % Z);
        g.echk.push_back(r * Z + i);
      }
      g.cptr.push_back(static_cast<int>(g.cvar.size()));
    }
  g.E = static_cast<int>(g.cvar.size());
  std::vector<int> deg(g.N, 0);
  for (int e = 0; e < g.E; ++e) deg[g.cvar[e]]++;
  g.vptr.assign(g.N + 1, 0);
  for (int v = 0; v < g.N; ++v) g.vptr[v + 1] = g.vptr[v] + deg[v];
  g.vedge.assign(g.E, 0);
  std::vector<int> fill(g.vptr.begin(), g.vptr.end() - 1);
  for (int e = 0; e < g.E; ++e) g.vedge[fill[g.cvar[e]]++] = e;  // edges are check-major
  return true;
}

template <class T>
int decode_batch(const Graph& g, int alg, const T* llr, int batch, int max_iter, int stop,
                 T alpha, uint8_t* hard, int32_t* iters, T* soft, uint8_t* flags,
                 int64_t* counts, int threads) {
  if (batch < 0 || max_iter < 1 || stop < 0 || stop > 2 || (stop == 2 && alg != CBP_SP) ||
      !llr || !hard || !iters)
    return -1;
  if (alg < 0 || alg > 5) return -1;
  if (alg == CBP_SP_OMEGA && sizeof(T) != sizeof(double)) return -1;
  if (threads < 1) threads = 1;
  threads = std::min(threads, std::max(batch, 1));
  std::vector<std::vector<int64_t>> cnt(threads, std::vector<int64_t>(C_COUNT, 0));
  auto work = [&](int tid) {
    Frame<T> f(g, cnt[tid].data());
    f.max_iter = max_iter;
    f.stop = stop;
    f.alpha = alpha;
    int lo = static_cast<int>(static_cast<int64_t>(batch) * tid / threads);
    int hi = static_cast<int>(static_cast<int64_t>(batch) * (tid + 1) / threads);
    for (int b = lo; b < hi; ++b) {
      f.L = llr + static_cast<int64_t>(b) * g.N;
      f.hard = hard + static_cast<int64_t>(b) * g.N;
      f.soft = soft ? soft + static_cast<int64_t>(b) * g.N : nullptr;
      f.flag = 0;
      f.iters = 0;
      switch (alg) {
        case CBP_SP: f.cbp_sp(); break;
        case CBP_NMS: f.cbp_nms(); break;
        case LBP_NMS: f.lbp(true); break;
        case FBP_SP: f.fbp(); break;
        case LBP_SP: f.lbp(false); break;
        case CBP_SP_OMEGA: f.cbp_sp_omega(); break;
      }
      iters[b] = f.iters;
      if (flags) flags[b] = f.flag;
    }
  };
  if (threads == 1) {
    work(0);
  } else {
    std::vector<std::thread> pool;
    for (int t = 0; t < threads; ++t) pool.emplace_back(work, t);
    for (auto& th : pool) th.join();
  }
  if (counts)
    for (int k = 0; k < C_COUNT; ++k) {
      counts[k] = 0;
      for (int t = 0; t < threads; ++t) counts[k] += cnt[t][k];
    }
  return 0;
}

}  // namespace

extern "C" {

struct orc_code {
  Graph g;
};

orc_code* orc_code_create(const int32_t* base, int mb, int nb, int Z) {
  orc_code* c = new orc_code;
  if (!build_graph(base, mb, nb, Z, c->g)) {
    delete c;
    return nullptr;
  }
  return c;
}

void orc_code_destroy(orc_code* c) { delete c; }

void orc_code_dims(const orc_code* c, int* N, int* M, int* E) {
  *N = c->g.N;
  *M = c->g.M;
  *E = c->g.E;
}

// Edge list of the expanded graph (check-major, ascending variable).
void orc_code_edges(const orc_code* c, int32_t* echk, int32_t* evar) {
  for (int e = 0; e < c->g.E; ++e) {
    echk[e] = c->g.echk[e];
    evar[e] = c->g.cvar[e];
  }
}

int orc_decode_f32(const orc_code* c, int alg, const float* llr, int batch, int max_iter, int stop,
                   float alpha, uint8_t* hard, int32_t* iters, float* soft, uint8_t* flags,
                   int64_t* counts, int threads) {
  if (!c) return -1;
  return decode_batch<float>(c->g, alg, llr, batch, max_iter, stop, alpha, hard, iters, soft,
                             flags, counts, threads);
}

int orc_decode_f64(const orc_code* c, int alg, const double* llr, int batch, int max_iter,
                   int stop, double alpha, uint8_t* hard, int32_t* iters, double* soft,
                   uint8_t* flags, int64_t* counts, int threads) {
  if (!c) return -1;
  return decode_batch<double>(c->g, alg, llr, batch, max_iter, stop, alpha, hard, iters, soft,
                              flags, counts, threads);
}

// CBP (S-domain, FP64) run for exactly `sweeps` sweeps on one frame; returns for every
// check its S = sum phi(|Q|) and sign, and for every edge the V2C message folded into
// that check at its latest visit, and the stored C2V message R.
int orc_cbp_trace_f64(const orc_code* c, const double* llr, int sweeps, double* S_out,
                      uint8_t* sig_out, double* q_edge, double* r_edge) {
  if (!c || sweeps < 1) return -1;
  const Graph& g = c->g;
  std::vector<double> Q(llr, llr + g.N), Ph(g.N, 0.0), S(g.M, 0.0), R(g.E, 0.0);
  std::vector<uint8_t> sg(g.M, 0);
  std::vector<int> last(g.N, -1);
  for (int t = 1; t <= sweeps; ++t)
    for (int m = 0; m < g.M; ++m) {
      double Sacc = 0.0;
      int sig = 0;
      for (int e = g.cptr[m]; e < g.cptr[m + 1]; ++e) {
        const int v = g.cvar[e];
        double Rn = 0.0;
        if (last[v] >= 0) {
          const int cj = g.echk[last[v]];
          Rn = sgn_apply(static_cast<bool>(sg[cj] ^ (Q[v] < 0.0)), phi64(std::fabs(S[cj] - Ph[v])));
          R[last[v]] = Rn;
        }
        double qn = (Q[v] + Rn) - R[e];
        double ph = phi64(std::fabs(qn));
        Sacc += ph;
        sig ^= (qn < 0.0);
        Q[v] = qn;
        Ph[v] = ph;
        last[v] = e;
        q_edge[e] = qn;
      }
      S[m] = Sacc;
      sg[m] = static_cast<uint8_t>(sig);
    }
  for (int m = 0; m < g.M; ++m) {
    S_out[m] = S[m];
    sig_out[m] = sg[m];
  }
  for (int e = 0; e < g.E; ++e) r_edge[e] = R[e];
  return 0;
}

// Weighted CBP forward (T sweeps, no stop) on `batch` frames: soft = flushed posterior.
int orc_weighted_f64(const orc_code* c, const double* llr, const double* w, int Tsw, int batch,
                     double* soft) {
  if (!c || Tsw < 1 || batch < 0) return -1;
  for (int b = 0; b < batch; ++b)
    weighted_forward<double>(c->g, llr + static_cast<int64_t>(b) * c->g.N, w, Tsw,
                             soft + static_cast<int64_t>(b) * c->g.N, nullptr, nullptr);
  return 0;
}

int orc_weighted_f32(const orc_code* c, const float* llr, const float* w, int Tsw, int batch,
                     float* soft) {
  if (!c || Tsw < 1 || batch < 0) return -1;
  for (int b = 0; b < batch; ++b)
    weighted_forward<float>(c->g, llr + static_cast<int64_t>(b) * c->g.N, w, Tsw,
                            soft + static_cast<int64_t>(b) * c->g.N, nullptr, nullptr);
  return 0;
}

// Reverse-mode adjoint of orc_weighted_f64: grad_w (T*mb, summed over the frames) and
// grad_llr ([batch][N]) from grad_soft = dLoss/dsoft ([batch][N]).  Overwrites both.
int orc_weighted_grad_f64(const orc_code* c, const double* llr, const double* w, int Tsw,
                          int batch, const double* grad_soft, double* grad_w, double* grad_llr) {
  if (!c || Tsw < 1 || batch < 0) return -1;
  const int N = c->g.N;
  std::fill(grad_w, grad_w + static_cast<size_t>(Tsw) * c->g.mb, 0.0);
  for (int b = 0; b < batch; ++b) {
    double* gl = grad_llr + static_cast<int64_t>(b) * N;
    std::fill(gl, gl + N, 0.0);
    weighted_backward(c->g, llr + static_cast<int64_t>(b) * N, w, Tsw,
                      grad_soft + static_cast<int64_t>(b) * N, grad_w, gl);
  }
  return 0;
}

void orc_phi_f32(const float* x, float* y, int64_t n) {
  for (int64_t i = 0; i < n; ++i) y[i] = phi32(x[i]);
}

void orc_phi_f64(const double* x, double* y, int64_t n) {
  for (int64_t i = 0; i < n; ++i) y[i] = phi64(x[i]);
}

int orc_phi_table_f32(float* out, int cap) {
  const PhiTable& t = phi_table();
  int n = static_cast<int>(t.c.size());
  if (out) std::memcpy(out, t.c.data(), sizeof(float) * std::min(n, cap));
  return n;
}

float orc_phi_xlo_f32(void) { return kXlo32; }
double orc_phi_xlo_f64(void) { return xlo64(); }

}  // extern "C"
