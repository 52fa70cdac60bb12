// libcbp host side: the C ABI of include/cbp.h, code tables, phi table, launch planning.
#include <algorithm>
#include <cmath>
#include <cstdlib>
#include <cstring>
#include <mutex>
#include <new>
#include <vector>

#include "cbp_internal.cuh"

namespace cbp {

// ---------------------------------------------------------------------------
// phi coefficient table.  For every grid centre m with normalisation h the cubic
// Taylor coefficients phi^(k)(m) h^k / k! are computed in FP64 from
//   phi(m) = log1p(2 / expm1(m)),  phi'(m) = -1/sinh m,  phi''(m) = cosh m / sinh^2 m,
//   phi'''(m) = -(1 + cosh^2 m) / sinh^3 m,
// and rounded to FP32.
// ---------------------------------------------------------------------------
void phi_table_host(float* coef, float* xlo) {
  for (int i = 0; i < kPhiSegments; ++i) {
    double m, h;
    if (i < kPhiLogCount) {
      uint32_t u = static_cast<uint32_t>(kPhiLogBase + i) << 18;
      float mf;
      std::memcpy(&mf, &u, sizeof mf);
      m = mf;
      int ex;
      std::frexp(m, &ex);      // m = f * 2^ex, f in [0.5, 1)
      h = std::ldexp(1.0, ex - 1);
    } else {
      m = static_cast<double>(i - kPhiLogCount + 32) / 16.0;
      h = 0.0625;
    }
    const double a = h / std::sinh(m);
    const double co = std::cosh(m);
    coef[4 * i + 0] = static_cast<float>(std::log1p(2.0 / std::expm1(m)));
    coef[4 * i + 1] = static_cast<float>(-a);
    coef[4 * i + 2] = static_cast<float>(0.5 * co * (a * a));
    coef[4 * i + 3] = static_cast<float>(-(co * co + 1.0) * (a * a * a) / 6.0);
  }
  *xlo = static_cast<float>(std::log1p(2.0 / std::expm1(30.0)));
}

// Coefficient k divided by h^k: h = 2^(e - 1) for a centre m = f 2^e (f in [0.5, 1)),
// h = 1/16 above 2.  ldexp by a power of two is exact while the value stays normal,
// which every coefficient does (the largest, |c3| / h^3 at m = 2^-43, is about 2^127.4).
void phi_table_device_form(const float* coef, float* dev) {
  for (int i = 0; i < kPhiSegments; ++i) {
    int lh;  // log2 h
    if (i < kPhiLogCount) {
      uint32_t u = static_cast<uint32_t>(kPhiLogBase + i) << 18;
      float mf;
      std::memcpy(&mf, &u, sizeof mf);
      int ex;
      std::frexp(static_cast<double>(mf), &ex);
      lh = ex - 1;
    } else {
      lh = -4;
    }
    for (int k = 0; k < 4; ++k) dev[4 * i + k] = std::ldexp(coef[4 * i + k], -k * lh);
  }
}

__device__ float4 g_phi_tab[kPhiSegments];

namespace {

constexpr int kMaxDevices = 64;

struct DeviceInfo {
  bool ready = false;
  int sms = 0;
  int smem_optin = 0;
  int smem_sm = 0;        // shared memory per SM
  float4* tab = nullptr;  // device address of g_phi_tab on this device
  float xlo = 0.0f;
};

std::mutex g_mu;
DeviceInfo g_dev[kMaxDevices];

int device_init(int dev, DeviceInfo** out) {
  if (dev < 0 || dev >= kMaxDevices) return CBP_EUNSUPPORTED;
  std::lock_guard<std::mutex> lk(g_mu);
  DeviceInfo& d = g_dev[dev];
  if (!d.ready) {
    static std::vector<float> coef;
    static float xlo = 0.0f;
    if (coef.empty()) {
      std::vector<float> t_form(4 * kPhiSegments);
      phi_table_host(t_form.data(), &xlo);
      coef.resize(4 * kPhiSegments);
      phi_table_device_form(t_form.data(), coef.data());
    }
    if (cudaMemcpyToSymbol(g_phi_tab, coef.data(), sizeof(float) * coef.size()) != cudaSuccess)
      return CBP_ECUDA;
    void* addr = nullptr;
    if (cudaGetSymbolAddress(&addr, g_phi_tab) != cudaSuccess) return CBP_ECUDA;
    if (cudaDeviceGetAttribute(&d.sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&d.smem_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) !=
            cudaSuccess ||
        cudaDeviceGetAttribute(&d.smem_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev) !=
            cudaSuccess)
      return CBP_ECUDA;
    const Variant all[] = {{ALG_CBP_SP, true, 1},  {ALG_CBP_SP, false, 1},
                           {ALG_CBP_SP, true, 2},  {ALG_CBP_SP, false, 2},
                           {ALG_CBP_SP, true, 1, true}, {ALG_CBP_SP, false, 1, true},
                           {ALG_CBP_SP, true, 1, false, true},
                           {ALG_CBP_SP, false, 1, false, true},
                           {ALG_CBP_SP, true, 1, false, false, true},
                           {ALG_CBP_SP, false, 1, false, false, true},
                           {ALG_CBP_SP, false, 1, false, false, false, true},
                           {ALG_CBP_SP, false, 1, false, false, false, false, false, true},
                           {ALG_CBP_SP, false, 1, false, false, false, false, false, true, true},
                           {ALG_LBP_NMS, false, 1, false, false, false, false, false, true},
                           {ALG_LBP_NMS, false, 1, false, false, false, false, false, true, true},
                           {ALG_CBP_NMS, false, 1, false, false, false, false, false, true},
                           {ALG_CBP_NMS, false, 1, false, false, false, false, false, true, true},
                           {ALG_CBP_NMS, true, 1}, {ALG_CBP_NMS, false, 1},
                           {ALG_CBP_NMS, true, 1, false, false, false, false, true},
                           {ALG_CBP_NMS, false, 1, false, false, false, false, true},
                           {ALG_LBP_NMS, false, 1}, {ALG_FBP_SP, false, 1}};
    for (const Variant& v : all)
      if (decoder_set_smem(v, d.smem_optin) != cudaSuccess) return CBP_ECUDA;
    for (int deg : {8, 16, kMaxDeg})  // the wavefront flooding kernel's degree buckets
      for (bool sh : {false, true}) {
        Variant v{ALG_FBP_SP, false, 1};
        v.lvl = true;
        v.shrec = sh;
        v.deg = deg;
        if (decoder_set_smem(v, d.smem_optin) != cudaSuccess) return CBP_ECUDA;
      }
    if (grad_set_smem(d.smem_optin) != cudaSuccess) return CBP_ECUDA;
    for (int chk = 0; chk < 2; ++chk)
      for (int fpt = 1; fpt <= 3; ++fpt) {  // 3: one frame per group, weight-1-last instance
        void* k = sp_multi_kernel_ptr(chk != 0, fpt == 3 ? 1 : fpt, fpt == 3);
        cudaFuncAttributes fa;
        if (cudaFuncGetAttributes(&fa, k) != cudaSuccess ||
            cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 d.smem_optin - static_cast<int>(fa.sharedSizeBytes)) !=
                cudaSuccess)
          return CBP_ECUDA;
      }
    d.tab = static_cast<float4*>(addr);
    d.xlo = xlo;
    d.ready = true;
  }
  *out = &d;
  return CBP_OK;
}

int current_device(DeviceInfo** out, int* dev_out) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return CBP_ECUDA;
  if (dev_out) *dev_out = dev;
  return device_init(dev, out);
}

}  // namespace

namespace {
size_t align4(size_t n) { return (n + 3) & ~static_cast<size_t>(3); }
size_t align64(size_t n) { return (n + 63) & ~static_cast<size_t>(63); }
}  // namespace

size_t shared_fixed_bytes(const Variant& v, const Shape& s, int groups) {
  size_t b = sizeof(BaseEdge) * s.nnzb + sizeof(int) * align4(s.mb + 1) +
             12 * align4(static_cast<size_t>(groups) * v.fpt);
  switch (v.alg) {
    case ALG_CBP_SP:  // SpEdge records in place of the BaseEdge list (same size)
      b += sizeof(float4) * kPhiSegments + sizeof(uint2) * ((s.nb + 1) & ~1);
      static_assert(sizeof(SpEdge) == sizeof(BaseEdge), "CBP-SP edge record size");
      break;
    case ALG_FBP_SP:
      b += sizeof(float4) * kPhiSegments + sizeof(ColEntry) * ((s.nnzb + 1) & ~1) +
           sizeof(int) * align4(s.nb + 1);
      break;
    default:  // min-sum kernels; CBP min-sum also the entries' per-lane form (SpEdge)
      b += (v.alg == ALG_CBP_NMS ? sizeof(SpEdge) * s.nnzb : 0) +
           sizeof(uint2) * ((s.nb + 1) & ~1);
  }
  return b;
}

size_t shared_frame_floats(const Variant& v, const Shape& s) {
  const size_t W = align4(s.words);
  switch (v.alg) {
    case ALG_CBP_SP:  // WIN: + window counter/stop (4 ints) + one ok byte per check lane
      return v.fpt * (2 * static_cast<size_t>(s.ncomp) * s.Z + (v.chk_shared ? align4(s.M) : 0) +
                      W) +
             (v.win ? 4 + align4((static_cast<size_t>(s.Z) + 3) / 4) : 0);
    case ALG_CBP_NMS:
      return align4(static_cast<size_t>(s.ncomp) * s.Z) +
             (v.chk_shared ? 2 * static_cast<size_t>((s.M + 1) & ~1) : 0) + W;
    case ALG_LBP_NMS:
      return align4(static_cast<size_t>(s.ncomp) * s.Z) + W;
    default:  // flooding: Lambda [N] | bits
      return align4(s.N) + W;
  }
}

WsLayout ws_layout(const Variant& v, const Shape& s) {
  WsLayout w;
  size_t f = 0;
  switch (v.alg) {
    case ALG_CBP_SP:  // R [E][fpt] | (Q*, phi) of weight-1 columns | S (not shared)
      f = align64(static_cast<size_t>(s.E) * v.fpt);
      w.off_sv = static_cast<long long>(f);
      f += align64(2 * static_cast<size_t>(v.fpt) * s.nself * s.Z);
      if (!v.chk_shared) {
        w.off_s = static_cast<long long>(f);
        f += align64(static_cast<size_t>(v.fpt) * s.M);
      }
      break;
    case ALG_CBP_NMS:
    case ALG_LBP_NMS:  // weight-1 column state | per-check state (uint4; with per-edge
                       // messages: R [E]) | CBP (min1, min2)
      w.off_sv = 0;
      f = align64(static_cast<size_t>(s.nself) * s.Z);
      w.off_s = static_cast<long long>(f);
      f += v.rstore ? align64(static_cast<size_t>(s.E)) : align64(4 * static_cast<size_t>(s.M));
      if (v.alg == ALG_CBP_NMS && !v.chk_shared) {
        w.off_c = static_cast<long long>(f);
        f += align64(2 * static_cast<size_t>(s.M));
      }
      break;
    default:  // flooding: R [E]
      f = align64(s.E);
  }
  w.slot = static_cast<long long>(f);  // multiple of 64 floats: 256-byte aligned groups
  return w;
}

}  // namespace cbp

using namespace cbp;

struct cbp_code {
  int dev = 0;
  int mb = 0, nb = 0, Z = 0, N = 0, M = 0, E = 0, K = -1, nnzb = 0, maxdeg = 0;
  int test_row = 0;          // a base row of the largest degree (the sweep-end pre-test)
  int ncomp = 0, nself = 0;  // columns of weight >= 2 / of weight 1
  bool self_last = true;     // every row holds at most one weight-1 entry, as its last
  int nlev = 0;              // levels of the wavefront schedule (0: tables not built)
  int lvl_maxw = 0;          // checks in its widest level
  int lvl_test = 0;          // that level
  CodeDev d;
  Shape shape() const {
    return Shape{Z, N, M, E, nnzb, mb, nb, (N + 31) / 32, ncomp, nself};
  }
};

namespace {

bool aligned(const void* p, size_t a) { return (reinterpret_cast<uintptr_t>(p) % a) == 0; }

// GF(2) rank of a small dense H (bit-packed rows).
int gf2_rank(const int32_t* base, int mb, int nb, int Z) {
  const int N = nb * Z, M = mb * Z, W = (N + 63) / 64;
  std::vector<uint64_t> h(static_cast<size_t>(M) * W, 0);
  for (int r = 0; r < mb; ++r)
    for (int i = 0; i < Z; ++i)
      for (int c = 0; c < nb; ++c) {
        int s = base[r * nb + c];
        if (s < 0) continue;
        int v = c * Z + (i + s) % Z;
        h[static_cast<size_t>(r * Z + i) * W + v / 64] ^= uint64_t(1) << (v % 64);
      }
  int rank = 0;
  for (int col = 0; col < N && rank < M; ++col) {
    const int w = col / 64;
    const uint64_t bit = uint64_t(1) << (col % 64);
    int piv = -1;
    for (int r = rank; r < M; ++r)
      if (h[static_cast<size_t>(r) * W + w] & bit) {
        piv = r;
        break;
      }
    if (piv < 0) continue;
    if (piv != rank)
      for (int k = 0; k < W; ++k)
        std::swap(h[static_cast<size_t>(piv) * W + k], h[static_cast<size_t>(rank) * W + k]);
    for (int r = 0; r < M; ++r)
      if (r != rank && (h[static_cast<size_t>(r) * W + w] & bit))
        for (int k = 0; k < W; ++k)
          h[static_cast<size_t>(r) * W + k] ^= h[static_cast<size_t>(rank) * W + k];
    ++rank;
  }
  return rank;
}

struct Plan {
  Variant v{};  // F below counts lane groups; a group decodes v.fpt frames
  int F = 0, threads = 0, grid = 0, ctas_per_sm = 0, frames_per_sm = 0;
  int team_groups = 0;  // lane groups per team (CBP-SP); >= F means one team
  size_t smem = 0;
  WsLayout ws{};
  int sh_frame = 0;
  size_t ws_bytes = 0;
  // frame-parallel kernel (v.fp): slots and workspace offsets, see KParams
  long long fp_slots = 0, fp_off_sv = 0, fp_off_s = 0, fp_off_r = 0, fp_off_b = 0;
  int lvl_lanes = 0;  // wavefront-schedule kernel (v.lvl): lanes per group
};

// CBP-SP takes the frame-parallel kernel when the lane-parallel plan keeps fewer lanes
// than this busy per SM (small Z with large per-frame shared state, e.g. Z = 1 codes), or
// when no frame fits its shared memory.
constexpr int kFpMinLanes = 128;

// Launch plan of the frame-parallel CBP-SP kernel: one frame slot per thread, as many
// CTAs as the SMs hold (fewer for small batches); the workspace holds each array of
// every slot element-major, slot innermost, each array 256-byte aligned.
int make_fp_plan(const cbp_code* c, const DeviceInfo& di, int batch, Plan* out) {
  Plan pl;
  pl.v = Variant{ALG_CBP_SP, false, 1};
  pl.v.fp = true;
  pl.threads = fp_threads();
  pl.smem = sizeof(float4) * kPhiSegments + sizeof(int) * align4(c->mb + 1) +
            sizeof(uint2) * ((c->nb + 1) & ~1);
  if (pl.smem > static_cast<size_t>(di.smem_optin)) return CBP_EUNSUPPORTED;
  int ctas = 0;
  if (decoder_occupancy(pl.v, pl.threads, pl.smem, &ctas) != cudaSuccess) return CBP_ECUDA;
  if (ctas < 1) return CBP_EUNSUPPORTED;
  const long long need = (static_cast<long long>(batch) + pl.threads - 1) / pl.threads;
  pl.grid = static_cast<int>(std::max(1LL, std::min<long long>(need, 1LL * di.sms * ctas)));
  pl.F = pl.threads;
  pl.team_groups = 1;
  pl.ctas_per_sm = ctas;
  pl.frames_per_sm = ctas * pl.threads;
  pl.fp_slots = static_cast<long long>(pl.grid) * pl.threads;
  long long off = 0;
  auto take = [&](long long elems) {
    const long long o = off;
    off += static_cast<long long>(align64(static_cast<size_t>(elems * pl.fp_slots)));
    return o;
  };
  take(2LL * c->ncomp * c->Z);  // QP at offset 0
  pl.fp_off_sv = take(2LL * c->nself * c->Z);
  pl.fp_off_s = take(c->M);
  pl.fp_off_r = take(c->E);
  pl.fp_off_b = take((c->N + 31) / 32);
  pl.ws_bytes = static_cast<size_t>(off) * sizeof(float);
  *out = pl;
  return CBP_OK;
}

// Launch plan of the wavefront-schedule kernel, one CTA per SM: as many lane groups (one
// frame each) as shared memory holds (CBP-SP: a frame's Q*, check-beliefs and decision bits;
// at most 15, one named barrier each), then the widest group of whole warps that keeps
// the CTA within its thread limit, but no wider than the widest level (CBP_LVL_LANES =
// 32..256 in the environment for tuning); fewer groups for small batches.  The workspace
// holds each group slot's C2V messages.  The edge records go to shared memory too when
// the code has the 8-byte form and a frame still fits (CBP_LVL_SHREC=0 keeps them in
// global memory).  Layered NMS (alg ALG_LBP_NMS): per frame Lambda and the check states
// instead, no phi table, no workspace, each edge's variable index in shared memory.  CBP
// min-sum (ALG_CBP_NMS): per frame Q* and (min1 | sgn, min2) per check, no phi table.
// Flooding (ALG_FBP_SP): per frame Lambda; the variables' edge lists in shared memory too.
int make_level_plan(const cbp_code* c, const DeviceInfo& di, int batch, Plan* out,
                    int alg = ALG_CBP_SP) {
  if (c->nlev == 0) return CBP_EUNSUPPORTED;
  const bool lbp = alg == ALG_LBP_NMS, nms = alg == ALG_CBP_NMS, fbp = alg == ALG_FBP_SP;
  if ((lbp || fbp) && c->maxdeg > kMaxDeg) return CBP_EUNSUPPORTED;
  Plan pl;
  pl.v = Variant{alg, false, 1};
  pl.v.lvl = true;
  size_t fixed = (lbp || nms ? 0 : sizeof(float4) * kPhiSegments) + sizeof(int) * 16;
  const size_t W = align4((static_cast<size_t>(c->N) + 31) / 32);
  const size_t fr_floats = lbp   ? 4 * static_cast<size_t>(c->M) + align4(c->N) + W
                           : nms ? 2 * static_cast<size_t>(c->M) + align4(c->N) + W
                           : fbp ? align4(c->N) + W
                                 : align4(c->N) + align4(c->M) + W;
  const size_t avail = static_cast<size_t>(di.smem_optin);
  const size_t recb = fbp ? sizeof(int) * (2 * align4(c->E) + align4(c->M + 1) + align4(c->N + 1))
                          : (lbp ? sizeof(uint32_t) * align4(c->E) : sizeof(uint2) * c->E) +
                                sizeof(int) * align4(c->M + 1);
  if (fbp) pl.v.deg = c->maxdeg <= 8 ? 8 : c->maxdeg <= 16 ? 16 : kMaxDeg;
  const char* es = std::getenv("CBP_LVL_SHREC");
  if ((lbp || fbp || c->d.lvl_rec8) && !(es && es[0] == '0') &&
      fixed + recb + fr_floats * 4 <= avail) {
    pl.v.shrec = true;
    fixed += recb;
  }
  if (fixed + fr_floats * 4 > avail) return CBP_EUNSUPPORTED;
  int F = static_cast<int>(std::min<size_t>((avail - fixed) / (fr_floats * 4), 15));
  // (flooding takes all checks at once, so the level widths do not bound its groups)
  int G = fbp ? 64
              : std::max(32, std::min((level_max_threads() / F) / 32 * 32,
                                      (c->lvl_maxw + 31) / 32 * 32));
  if (const char* e = std::getenv("CBP_LVL_LANES")) {
    const int g = std::atoi(e);
    if (g >= 32 && g <= 256 && g % 32 == 0) G = g;
  }
  F = std::min(F, level_max_threads() / G);
  const int spread = std::max(1, (batch + di.sms - 1) / di.sms);
  F = std::max(1, std::min(F, spread));
  pl.F = F;
  pl.threads = F * G;
  pl.smem = fixed + static_cast<size_t>(F) * fr_floats * 4;
  int ctas = 0;
  if (decoder_occupancy(pl.v, pl.threads, pl.smem, &ctas) != cudaSuccess) return CBP_ECUDA;
  if (ctas < 1) return CBP_EUNSUPPORTED;
  const long long need = (static_cast<long long>(batch) + F - 1) / F;
  pl.grid = static_cast<int>(std::max(1LL, std::min<long long>(need, 1LL * di.sms * ctas)));
  pl.team_groups = 1;
  pl.ctas_per_sm = ctas;
  pl.frames_per_sm = ctas * F;
  pl.sh_frame = static_cast<int>(fr_floats);
  pl.lvl_lanes = G;
  pl.ws.slot = lbp ? 0 : static_cast<long long>(align64(static_cast<size_t>(c->E)));
  pl.ws_bytes = static_cast<size_t>(pl.grid) * F * static_cast<size_t>(pl.ws.slot) * sizeof(float);
  *out = pl;
  return CBP_OK;
}

// Lane groups per team (CBP-SP and min-sum kernels): the smallest multiple of the
// groups that fill whole warps which splits the CTA into 2..15 equal teams (named
// barriers 1..15); otherwise the whole CTA is one team.
int team_groups_for(int Z, int groups) {
  int a = Z, b = 32;
  while (b) {
    const int r = a % b;
    a = b;
    b = r;
  }
  for (int tg = 32 / a; tg <= groups / 2; tg += 32 / a)
    if (groups % tg == 0 && groups / tg <= 15) return tg;
  return groups;
}

// Launch plan: for each layout variant the number of lane groups per CTA that gives the
// most resident frames per SM (ties: more resident warps); the variant with the most
// resident frames wins (ties: the earlier one in the candidate list).  CBP_PLAN_CHK=0/1
// and CBP_PLAN_FPT=1/2 in the environment restrict the candidates (tuning experiments).
int make_lane_plan(const cbp_code* c, const DeviceInfo& di, int alg, int batch, Plan* out,
                   int stop) {
  std::vector<Variant> cands;
  switch (alg) {
    case ALG_CBP_SP:
      if (stop == CBP_STOP_WINDOW) {  // one frame per group, row degree <= 32 (flip masks)
        if (c->Z > 384 || c->maxdeg > 32) return CBP_EUNSUPPORTED;
        cands = {{ALG_CBP_SP, true, 1, false, true}, {ALG_CBP_SP, false, 1, false, true}};
        break;
      }
      cands = {{ALG_CBP_SP, true, 2}, {ALG_CBP_SP, false, 2},
               {ALG_CBP_SP, true, 1, false, false, c->self_last},
               {ALG_CBP_SP, false, 1, false, false, c->self_last}};
      if (c->Z > 384) cands.push_back({ALG_CBP_SP, true, 1, true});
      if (c->Z > 384) cands.push_back({ALG_CBP_SP, false, 1, true});
      break;
    case ALG_CBP_NMS:
      if (c->maxdeg > kMaxDegCbpMs) return CBP_EUNSUPPORTED;
      cands = {{ALG_CBP_NMS, true}, {ALG_CBP_NMS, false}};
      if (const char* e = std::getenv("CBP_PLAN_NMS_R"); e && e[0] == '1')
        for (Variant& v : cands) v.rstore = true;
      break;
    case ALG_LBP_NMS:
      if (c->maxdeg > kMaxDeg) return CBP_EUNSUPPORTED;
      cands = {{ALG_LBP_NMS, false}};
      break;
    case ALG_FBP_SP:
      if (c->maxdeg > kMaxDeg) return CBP_EUNSUPPORTED;
      cands = {{ALG_FBP_SP, false}};
      break;
    default:
      return CBP_EINVAL;
  }
  if (const char* e = std::getenv("CBP_PLAN_CHK")) {
    if (alg == ALG_CBP_SP || alg == ALG_CBP_NMS) {
      const bool want = e[0] == '1';
      cands.erase(std::remove_if(cands.begin(), cands.end(),
                                 [&](const Variant& v) { return v.chk_shared != want; }),
                  cands.end());
    }
  }
  if (const char* e = std::getenv("CBP_PLAN_FPT")) {
    const int want = e[0] == '2' ? 2 : 1;
    cands.erase(std::remove_if(cands.begin(), cands.end(),
                               [&](const Variant& v) { return v.fpt != want; }),
                cands.end());
  }
  const Shape sh = c->shape();
  bool found = false;
  Plan best;
  int best_frames = -1, best_warps = -1, best_ctas = 0;
  for (const Variant& v : cands) {
    cudaFuncAttributes fa;
    if (decoder_func_attrs(v, &fa) != cudaSuccess) return CBP_ECUDA;
    const int fmax = fa.maxThreadsPerBlock / c->Z;
    const size_t fr_floats = shared_frame_floats(v, sh);
    for (int F = 1; F <= fmax; ++F) {
      const size_t smem = shared_fixed_bytes(v, sh, F) + F * fr_floats * 4;
      if (smem > static_cast<size_t>(di.smem_optin)) break;
      const int threads = (F * c->Z + 31) / 32 * 32;
      if (threads > fa.maxThreadsPerBlock) break;
      int ctas = 0;
      if (decoder_occupancy(v, threads, smem, &ctas) != cudaSuccess) return CBP_ECUDA;
      const int warps = ctas * threads / 32;
      const int frames = ctas * F * v.fpt;
      if (ctas >= 1 && (frames > best_frames || (frames == best_frames && warps > best_warps))) {
        best_frames = frames;
        best_warps = warps;
        best_ctas = ctas;
        best.v = v;
        best.F = F;
        best.threads = threads;
        best.smem = smem;
        best.sh_frame = static_cast<int>(fr_floats);
        found = true;
      }
    }
  }
  if (!found) return CBP_EUNSUPPORTED;
  // small batches: fewer lane groups per CTA so the frames spread over the SMs
  const int per_group = best.v.fpt;
  const int spread = std::max(1, (batch + di.sms * per_group - 1) / (di.sms * per_group));
  if (best.F > spread) {
    best.F = spread;
    best.threads = (best.F * c->Z + 31) / 32 * 32;
    best.smem = shared_fixed_bytes(best.v, sh, best.F) +
                best.F * static_cast<size_t>(best.sh_frame) * 4;
  }
  best.team_groups = team_groups_for(c->Z, best.F);
  best.ctas_per_sm = best_ctas;
  best.frames_per_sm = best_frames;
  const long long per_cta = static_cast<long long>(best.F) * per_group;
  const long long need = (static_cast<long long>(batch) + per_cta - 1) / per_cta;
  best.grid = static_cast<int>(std::max(1LL, std::min<long long>(need, 1LL * di.sms * best_ctas)));
  best.ws = ws_layout(best.v, sh);
  best.ws_bytes = static_cast<size_t>(best.grid) * best.F * best.ws.slot * sizeof(float);
  *out = best;
  return CBP_OK;
}

// Launch plan of a decode: the lane-parallel kernels, or for CBP-SP the frame-parallel one
// where the lane-parallel plan would leave the SMs' lanes idle (CBP_PLAN_FP=0/1 in the
// environment forces either; the paper-literal stop and the no-alloc entry point always
// run lane-parallel).
// CBP-SP where the lane-parallel plan keeps fewer than kFpMinLanes lanes per SM busy (or
// has none): the wavefront-schedule kernel when its tables exist and a frame fits, else
// the frame-parallel kernel.  CBP_PLAN_FP=1 / CBP_PLAN_LEVEL=1 force one of them,
// CBP_PLAN_FP=0 keeps the lane-parallel plan, CBP_PLAN_LEVEL=0 skips the wavefront kernel.
int make_plan(const cbp_code* c, const DeviceInfo& di, int alg, int batch, Plan* out,
              int stop = CBP_STOP_SYNDROME, bool allow_fp = true) {
  if ((alg == ALG_LBP_NMS || alg == ALG_CBP_NMS || alg == ALG_FBP_SP) && allow_fp) {
    // the same choice for the comparators, which have no frame-parallel kernel
    const char* el = std::getenv("CBP_PLAN_LEVEL");
    if (el && el[0] == '1') return make_level_plan(c, di, batch, out, alg);
    const int rc = make_lane_plan(c, di, alg, batch, out, stop);
    if (!(el && el[0] == '0') &&
        (rc == CBP_EUNSUPPORTED || (rc == CBP_OK && 1LL * out->frames_per_sm * c->Z < kFpMinLanes))) {
      Plan lp;
      if (make_level_plan(c, di, batch, &lp, alg) == CBP_OK) {
        *out = lp;
        return CBP_OK;
      }
    }
    return rc;
  }
  const bool sp = alg == ALG_CBP_SP && stop != CBP_STOP_WINDOW && allow_fp;
  const char* e = sp ? std::getenv("CBP_PLAN_FP") : nullptr;
  const char* el = sp ? std::getenv("CBP_PLAN_LEVEL") : nullptr;
  if (e && e[0] == '1') return make_fp_plan(c, di, batch, out);
  if (el && el[0] == '1') return make_level_plan(c, di, batch, out);
  const int rc = make_lane_plan(c, di, alg, batch, out, stop);
  if (!sp || (e && e[0] == '0')) return rc;
  if (rc == CBP_EUNSUPPORTED ||
      (rc == CBP_OK && 1LL * out->frames_per_sm * c->Z < kFpMinLanes)) {
    Plan lp;
    if (!(el && el[0] == '0') && make_level_plan(c, di, batch, &lp) == CBP_OK) {
      *out = lp;
      return CBP_OK;
    }
    return make_fp_plan(c, di, batch, out);
  }
  return rc;
}

// Kernel parameters of one code under a plan (buffers are filled in by the caller).
KParams code_params(const cbp_code* c, const DeviceInfo& di, const Plan& pl, int batch,
                    int max_iter, int stop, float alpha) {
  KParams p{};
  p.status = c->d.status;
  p.edges = c->d.edges;
  p.spe = c->d.spe;
  p.rptr = c->d.rptr;
  p.cols = c->d.cols;
  p.cptr = c->d.cptr;
  p.phi_tab = di.tab;
  p.phi_xlo = di.xlo;
  p.Z = c->Z;
  p.mb = c->mb;
  p.nb = c->nb;
  p.nnzb = c->nnzb;
  p.N = c->N;
  p.M = c->M;
  p.E = c->E;
  p.words = (c->N + 31) / 32;
  p.batch = batch;
  p.max_iter = max_iter;
  p.stop = stop;
  p.alpha = alpha;
  p.F = pl.F;
  p.team_groups = team_groups_for(c->Z, pl.F);
  p.slots = pl.grid * pl.F * pl.v.fpt;
  p.maxdeg = c->maxdeg;
  p.test_row = c->test_row;
  p.ncomp = c->ncomp;
  p.nself = c->nself;
  p.ws_slot = pl.ws.slot;
  p.ws_off_sv = pl.ws.off_sv;
  p.ws_off_s = pl.ws.off_s;
  p.ws_off_c = pl.ws.off_c;
  p.ws_cta = static_cast<long long>(pl.F) * pl.ws.slot;
  p.sh_frame = pl.sh_frame;
  p.fp_slots = pl.fp_slots;
  p.fp_off_sv = pl.fp_off_sv;
  p.fp_off_s = pl.fp_off_s;
  p.fp_off_r = pl.fp_off_r;
  p.fp_off_b = pl.fp_off_b;
  p.lvl_ptr = c->d.lvl_ptr;
  p.lvl_e0 = c->d.lvl_e0;
  p.lvl_edge = c->d.lvl_edge;
  p.lvl_rec8 = c->d.lvl_rec8;
  p.last_chk = c->d.last_chk;
  p.lvl_cptr = c->d.lvl_cptr;
  p.lvl_cedge = c->d.lvl_cedge;
  p.nlev = c->nlev;
  p.lvl_lanes = pl.lvl_lanes;
  p.lvl_test = c->lvl_test;
  return p;
}

int check_opts(const cbp_opts_t* o, int* alg, float* alpha, int* stop, float** soft) {
  *alg = CBP_ALG_CBP_SP;
  *alpha = 0.75f;
  *stop = CBP_STOP_SYNDROME;
  *soft = nullptr;
  if (!o) return CBP_OK;
  if (o->alg < CBP_ALG_CBP_SP || o->alg > CBP_ALG_FBP_SP) return CBP_EINVAL;
  if (o->stop_mode != CBP_STOP_SYNDROME && o->stop_mode != CBP_STOP_NONE &&
      o->stop_mode != CBP_STOP_WINDOW)
    return CBP_EINVAL;
  if (o->stop_mode == CBP_STOP_WINDOW && (o->alg != CBP_ALG_CBP_SP || o->soft_out))
    return CBP_EINVAL;
  if (!std::isfinite(o->alpha)) return CBP_EINVAL;
  *alg = o->alg;
  if (o->alpha > 0.0f) *alpha = o->alpha;
  *stop = o->stop_mode;
  *soft = o->soft_out;
  if (*soft && !aligned(*soft, 4)) return CBP_EINVAL;
  return CBP_OK;
}

// Largest expanded edge count for which the wavefront schedule is built (16 MB of records).
constexpr long long kLvlMaxEdges = 1 << 20;

// The wavefront schedule of the expanded graph: checks m = r*Z + z in the paper's order,
// the variables of a check in ascending base column.  level(m) = 1 + the largest level of
// the previous check (in that order) of each of m's variables, 0 if there is none; checks
// are listed by level, then index, and their edges renumbered in that order.
int build_level_tables(cbp_code* c, const std::vector<BaseEdge>& edges,
                       const std::vector<int>& rptr) {
  const int Z = c->Z, M = c->M, N = c->N, E = c->E;
  std::vector<int> ep(M + 1, 0), ev(E), echk(E);
  std::vector<int> colw(c->nb, 0);
  for (const BaseEdge& be : edges) ++colw[be.c];
  for (int r = 0, e = 0; r < c->mb; ++r)
    for (int z = 0; z < Z; ++z) {
      const int m = r * Z + z;
      ep[m] = e;
      for (int k = rptr[r]; k < rptr[r + 1]; ++k) {
        ev[e] = edges[k].c * Z + (z + edges[k].s) % Z;
        echk[e] = m;
        ++e;
      }
      ep[m + 1] = e;
    }
  std::vector<int> level(M, 0), pred(E, -1), last_e(N, -1);
  int nlev = 0;
  for (int m = 0; m < M; ++m) {
    int lv = 0;
    for (int e = ep[m]; e < ep[m + 1]; ++e)
      if (last_e[ev[e]] >= 0) lv = std::max(lv, level[echk[last_e[ev[e]]]] + 1);
    level[m] = lv;
    nlev = std::max(nlev, lv + 1);
    for (int e = ep[m]; e < ep[m + 1]; ++e) {
      pred[e] = last_e[ev[e]];
      last_e[ev[e]] = e;
    }
  }
  std::vector<int> lptr(nlev + 1, 0), order(M), newidx(E);
  for (int m = 0; m < M; ++m) ++lptr[level[m] + 1];
  for (int l = 0; l < nlev; ++l)
    if (lptr[l + 1] > c->lvl_maxw) {
      c->lvl_maxw = lptr[l + 1];
      c->lvl_test = l;
    }
  for (int l = 0; l < nlev; ++l) lptr[l + 1] += lptr[l];
  {
    std::vector<int> fill(lptr.begin(), lptr.end() - 1);
    for (int m = 0; m < M; ++m) order[fill[level[m]]++] = m;
  }
  std::vector<int> e0(M + 1), cpos(M);
  for (int ci = 0, e2 = 0; ci < M; ++ci) {
    const int m = order[ci];
    cpos[m] = ci;
    e0[ci] = e2;
    for (int e = ep[m]; e < ep[m + 1]; ++e) newidx[e] = e2++;
  }
  e0[M] = E;
  const bool small = M <= 4096 && E < (1 << 20);  // the 8-byte record form
  std::vector<LvlEdge> rec(E);
  std::vector<uint2> rec8(small ? E : 0);
  for (int e = 0; e < E; ++e) {
    const int v = ev[e];
    const bool first = pred[e] < 0;
    const int pe = first ? last_e[v] : pred[e];  // cyclically: the last check of v
    const uint32_t x = static_cast<uint32_t>(v) | (first ? kSpFirst : 0u) |
                       (colw[v / Z] == 1 ? kSpSelf : 0u);
    const uint32_t cj = static_cast<uint32_t>(cpos[echk[pe]]);
    const uint32_t pn = static_cast<uint32_t>(newidx[pe]);
    rec[newidx[e]] = make_uint4(x, cj, pn, 0u);
    if (small) rec8[newidx[e]] = make_uint2(x, pn | (cj << 20));
  }
  std::vector<int> lastc(N);
  for (int v = 0; v < N; ++v) lastc[v] = cpos[echk[last_e[v]]];
  std::vector<int> cptr(N + 1, 0), cedge(E);  // each variable's edges, ascending check
  for (int e = 0; e < E; ++e) ++cptr[ev[e] + 1];
  for (int v = 0; v < N; ++v) cptr[v + 1] += cptr[v];
  {
    std::vector<int> fill(cptr.begin(), cptr.end() - 1);
    for (int e = 0; e < E; ++e) cedge[fill[ev[e]]++] = newidx[e];  // e ascends with the check
  }
  bool ok = cudaMalloc(&c->d.lvl_ptr, sizeof(int) * lptr.size()) == cudaSuccess &&
            cudaMalloc(&c->d.lvl_e0, sizeof(int) * e0.size()) == cudaSuccess &&
            cudaMalloc(&c->d.lvl_edge, sizeof(LvlEdge) * rec.size()) == cudaSuccess &&
            (!small || cudaMalloc(&c->d.lvl_rec8, sizeof(uint2) * rec8.size()) == cudaSuccess) &&
            cudaMalloc(&c->d.last_chk, sizeof(int) * lastc.size()) == cudaSuccess &&
            cudaMalloc(&c->d.lvl_cptr, sizeof(int) * cptr.size()) == cudaSuccess &&
            cudaMalloc(&c->d.lvl_cedge, sizeof(int) * cedge.size()) == cudaSuccess;
  if (!ok) return CBP_ENOMEM;
  ok = cudaMemcpy(c->d.lvl_ptr, lptr.data(), sizeof(int) * lptr.size(),
                  cudaMemcpyHostToDevice) == cudaSuccess &&
       cudaMemcpy(c->d.lvl_e0, e0.data(), sizeof(int) * e0.size(), cudaMemcpyHostToDevice) ==
           cudaSuccess &&
       cudaMemcpy(c->d.lvl_edge, rec.data(), sizeof(LvlEdge) * rec.size(),
                  cudaMemcpyHostToDevice) == cudaSuccess &&
       (!small || cudaMemcpy(c->d.lvl_rec8, rec8.data(), sizeof(uint2) * rec8.size(),
                             cudaMemcpyHostToDevice) == cudaSuccess) &&
       cudaMemcpy(c->d.last_chk, lastc.data(), sizeof(int) * lastc.size(),
                  cudaMemcpyHostToDevice) == cudaSuccess &&
       cudaMemcpy(c->d.lvl_cptr, cptr.data(), sizeof(int) * cptr.size(),
                  cudaMemcpyHostToDevice) == cudaSuccess &&
       cudaMemcpy(c->d.lvl_cedge, cedge.data(), sizeof(int) * cedge.size(),
                  cudaMemcpyHostToDevice) == cudaSuccess;
  if (!ok) return CBP_ECUDA;
  c->nlev = nlev;
  return CBP_OK;
}

}  // namespace

extern "C" {

int cbp_code_create(const int32_t* base, int mb, int nb, int Z, cbp_code_t** out) {
  if (!base || !out || mb < 1 || nb < 1 || Z < 1) return CBP_EINVAL;
  for (long long i = 0; i < 1LL * mb * nb; ++i)
    if (base[i] < -1 || base[i] >= Z) return CBP_EINVAL;
  int nnzb = 0, maxdeg = 0;
  for (int r = 0; r < mb; ++r) {
    int d = 0;
    for (int c = 0; c < nb; ++c) d += base[r * nb + c] >= 0;
    if (d < 2) return CBP_EINVAL;
    nnzb += d;
    maxdeg = std::max(maxdeg, d);
  }
  for (int c = 0; c < nb; ++c) {
    int w = 0;
    for (int r = 0; r < mb; ++r) w += base[r * nb + c] >= 0;
    if (w < 1) return CBP_EINVAL;
  }
  if (Z > 1024 || mb > 4096 || nb > 4096 || nnzb > 65535) return CBP_EUNSUPPORTED;
  if (1LL * nb * Z > (1LL << 30) / 4) return CBP_EUNSUPPORTED;

  DeviceInfo* di = nullptr;
  int dev = 0;
  if (int rc = current_device(&di, &dev)) return rc;

  // row-major entry list with each entry's predecessor in its column
  std::vector<int> idx(static_cast<size_t>(mb) * nb, -1);
  std::vector<BaseEdge> edges;
  std::vector<int> rptr(1, 0);
  for (int r = 0; r < mb; ++r) {
    for (int c = 0; c < nb; ++c)
      if (base[r * nb + c] >= 0) {
        idx[r * nb + c] = static_cast<int>(edges.size());
        BaseEdge e{};
        e.c = static_cast<uint16_t>(c);
        e.s = static_cast<uint16_t>(base[r * nb + c]);
        edges.push_back(e);
      }
    rptr.push_back(static_cast<int>(edges.size()));
  }
  std::vector<ColEntry> cols;
  std::vector<int> cptr(1, 0);
  int ncomp = 0, nself = 0;
  for (int c = 0; c < nb; ++c) {
    std::vector<int> rows;
    for (int r = 0; r < mb; ++r)
      if (base[r * nb + c] >= 0) rows.push_back(r);
    const int w = static_cast<int>(rows.size());
    const uint32_t kind_idx = static_cast<uint32_t>(w == 1 ? nself++ : ncomp++);
    for (int k = 0; k < w; ++k) {
      const int r = rows[k], pr = rows[(k + w - 1) % w];
      BaseEdge& e = edges[idx[r * nb + c]];
      e.pr = static_cast<uint16_t>(pr);
      e.ps = static_cast<uint16_t>(base[pr * nb + c]);
      e.pe = static_cast<uint16_t>(idx[pr * nb + c]);
      e.flags = static_cast<uint16_t>((k == 0 ? kFirst : 0) | (w == 1 ? kSelf : 0) |
                                      (k == w - 1 ? kLast : 0));
      e.pad = kind_idx;
      ColEntry ce{};
      ce.r = static_cast<uint16_t>(r);
      ce.s = static_cast<uint16_t>(base[r * nb + c]);
      ce.e = static_cast<uint16_t>(idx[r * nb + c]);
      cols.push_back(ce);
    }
    cptr.push_back(static_cast<int>(cols.size()));
  }

  cbp_code* c = new (std::nothrow) cbp_code;
  if (!c) return CBP_ENOMEM;
  for (int r = 0; r < mb && c->self_last; ++r)
    for (int k = rptr[r]; k < rptr[r + 1]; ++k)
      if ((edges[k].flags & kSelf) && k != rptr[r + 1] - 1) c->self_last = false;
  c->dev = dev;
  c->mb = mb;
  c->nb = nb;
  c->Z = Z;
  c->N = nb * Z;
  c->M = mb * Z;
  c->nnzb = nnzb;
  c->E = nnzb * Z;
  c->maxdeg = maxdeg;
  for (int r = 0; r < mb; ++r)
    if (rptr[r + 1] - rptr[r] == maxdeg) {
      c->test_row = r;
      break;
    }
  c->ncomp = ncomp;
  c->nself = nself;
  // K = N - rank(H): full rank when the parity part is block lower-triangular with
  // an identity-shift diagonal in column (nb - mb + r); else eliminate small codes.
  bool tri = nb > mb;
  for (int r = 0; r < mb && tri; ++r) {
    const int p = nb - mb + r;
    if (base[r * nb + p] < 0) tri = false;
    for (int cc = p + 1; cc < nb && tri; ++cc)
      if (base[r * nb + cc] >= 0) tri = false;
  }
  if (tri) c->K = c->N - c->M;
  else if (1LL * c->M * c->N <= (1LL << 24)) c->K = c->N - gf2_rank(base, mb, nb, Z);

  std::vector<SpEdge> spe(edges.size());
  for (size_t k = 0; k < edges.size(); ++k) {
    const BaseEdge& e = edges[k];
    const bool self = e.flags & kSelf;
    const uint32_t sq = self ? 0u : e.s;
    const uint32_t d = (static_cast<uint32_t>(e.s) + Z - e.ps) % static_cast<uint32_t>(Z);
    spe[k].x = ((e.pad & 0xffffu) * static_cast<uint32_t>(Z) + sq) |
               ((e.flags & kFirst) ? kSpFirst : 0u) | (self ? kSpSelf : 0u);
    spe[k].y = static_cast<uint32_t>(e.pr) * Z + d;
    spe[k].z = static_cast<uint32_t>(e.pe) * Z + d;
    spe[k].w = (static_cast<uint32_t>(Z) - sq) | ((static_cast<uint32_t>(Z) - d) << 16);
  }
  bool ok = cudaMalloc(&c->d.status, 2 * sizeof(uint32_t)) == cudaSuccess &&
            cudaMalloc(&c->d.edges, sizeof(BaseEdge) * edges.size()) == cudaSuccess &&
            cudaMalloc(&c->d.spe, sizeof(SpEdge) * spe.size()) == cudaSuccess &&
            cudaMalloc(&c->d.rptr, sizeof(int) * rptr.size()) == cudaSuccess &&
            cudaMalloc(&c->d.cols, sizeof(ColEntry) * cols.size()) == cudaSuccess &&
            cudaMalloc(&c->d.cptr, sizeof(int) * cptr.size()) == cudaSuccess;
  if (!ok) {
    cbp_code_destroy(c);
    return CBP_ENOMEM;
  }
  ok = cudaMemset(c->d.status, 0, 2 * sizeof(uint32_t)) == cudaSuccess &&
       cudaMemcpy(c->d.edges, edges.data(), sizeof(BaseEdge) * edges.size(),
                  cudaMemcpyHostToDevice) == cudaSuccess &&
       cudaMemcpy(c->d.spe, spe.data(), sizeof(SpEdge) * spe.size(), cudaMemcpyHostToDevice) ==
           cudaSuccess &&
       cudaMemcpy(c->d.rptr, rptr.data(), sizeof(int) * rptr.size(), cudaMemcpyHostToDevice) ==
           cudaSuccess &&
       cudaMemcpy(c->d.cols, cols.data(), sizeof(ColEntry) * cols.size(),
                  cudaMemcpyHostToDevice) == cudaSuccess &&
       cudaMemcpy(c->d.cptr, cptr.data(), sizeof(int) * cptr.size(), cudaMemcpyHostToDevice) ==
           cudaSuccess;
  if (!ok) {
    cbp_code_destroy(c);
    return CBP_ECUDA;
  }
  if (1LL * nnzb * Z <= kLvlMaxEdges) {
    if (int rc = build_level_tables(c, edges, rptr)) {
      cbp_code_destroy(c);
      return rc;
    }
  }
  *out = c;
  return CBP_OK;
}

void cbp_code_destroy(cbp_code_t* c) {
  if (!c) return;
  cudaFree(c->d.status);
  cudaFree(c->d.edges);
  cudaFree(c->d.spe);
  cudaFree(c->d.rptr);
  cudaFree(c->d.cols);
  cudaFree(c->d.cptr);
  cudaFree(c->d.lvl_ptr);
  cudaFree(c->d.lvl_e0);
  cudaFree(c->d.lvl_edge);
  cudaFree(c->d.lvl_rec8);
  cudaFree(c->d.last_chk);
  cudaFree(c->d.lvl_cptr);
  cudaFree(c->d.lvl_cedge);
  delete c;
}

int cbp_code_info(const cbp_code_t* c, int* n, int* m, int* k, int* edges) {
  if (!c) return CBP_EINVAL;
  if (n) *n = c->N;
  if (m) *m = c->M;
  if (k) *k = c->K;
  if (edges) *edges = c->E;
  return CBP_OK;
}

int cbp_workspace_bytes(const cbp_code_t* c, int batch, const cbp_opts_t* opts, size_t* bytes) {
  if (!c || !bytes || batch < 0) return CBP_EINVAL;
  int alg, stop;
  float alpha;
  float* soft;
  if (int rc = check_opts(opts, &alg, &alpha, &stop, &soft)) return rc;
  if (batch == 0) {
    *bytes = 0;
    return CBP_OK;
  }
  DeviceInfo* di = nullptr;
  int dev = 0;
  if (int rc = current_device(&di, &dev)) return rc;
  if (dev != c->dev) return CBP_EDEVICE;
  Plan pl;
  if (int rc = make_plan(c, *di, alg, batch, &pl, stop)) return rc;
  *bytes = pl.ws_bytes;
  return CBP_OK;
}

int cbp_launch_info(const cbp_code_t* c, int batch, const cbp_opts_t* opts, int* info) {
  if (!c || !info || batch < 1) return CBP_EINVAL;
  int alg, stop;
  float alpha;
  float* soft;
  if (int rc = check_opts(opts, &alg, &alpha, &stop, &soft)) return rc;
  DeviceInfo* di = nullptr;
  int dev = 0;
  if (int rc = current_device(&di, &dev)) return rc;
  if (dev != c->dev) return CBP_EDEVICE;
  Plan pl;
  if (int rc = make_plan(c, *di, alg, batch, &pl, stop)) return rc;
  info[0] = pl.frames_per_sm;
  info[1] = pl.threads;
  info[2] = pl.ctas_per_sm;
  info[3] = pl.F;
  info[4] = pl.v.fpt;
  info[5] = pl.v.chk_shared ? 1 : 0;
  info[6] = pl.grid;
  info[7] = pl.team_groups;
  info[8] = static_cast<int>(pl.smem);
  info[9] = pl.v.self_last ? 1 : 0;
  info[10] = pl.v.fp ? 1 : 0;
  info[11] = pl.v.lvl ? 1 : 0;
  return CBP_OK;
}

int cbp_decode_ex(const cbp_code_t* c, const float* llr, uint32_t* hard_out, int32_t* iters_out,
                  int max_iter, int batch, void* workspace, size_t workspace_bytes,
                  cbp_stream_t stream, const cbp_opts_t* opts) {
  if (!c || max_iter < 1 || batch < 0) return CBP_EINVAL;
  int alg, stop;
  float alpha;
  float* soft;
  if (int rc = check_opts(opts, &alg, &alpha, &stop, &soft)) return rc;
  if (batch == 0) return CBP_OK;
  if (!llr || !hard_out || !iters_out || !workspace) return CBP_EINVAL;
  if (!aligned(llr, 16) || !aligned(hard_out, 4) || !aligned(iters_out, 4) ||
      !aligned(workspace, 256))
    return CBP_EINVAL;
  DeviceInfo* di = nullptr;
  int dev = 0;
  if (int rc = current_device(&di, &dev)) return rc;
  if (dev != c->dev) return CBP_EDEVICE;
  Plan pl;
  if (int rc = make_plan(c, *di, alg, batch, &pl, stop)) return rc;
  if (workspace_bytes < pl.ws_bytes) return CBP_EWORKSPACE;

  KParams p = code_params(c, *di, pl, batch, max_iter, stop, alpha);
  p.llr = llr;
  p.hard = hard_out;
  p.iters = iters_out;
  p.soft = soft;
  p.ws = static_cast<float*>(workspace);
  cudaError_t e = launch_decoder(pl.v, p, pl.grid, pl.threads, pl.smem,
                                 reinterpret_cast<cudaStream_t>(stream));
  return e == cudaSuccess ? CBP_OK : CBP_ECUDA;
}

int cbp_decode(const cbp_code_t* c, const float* llr, uint32_t* hard_out, int32_t* iters_out,
               int max_iter, int batch, void* workspace, size_t workspace_bytes,
               cbp_stream_t stream) {
  return cbp_decode_ex(c, llr, hard_out, iters_out, max_iter, batch, workspace,
                       workspace_bytes, stream, nullptr);
}

// ---------------------------------------------------------------------------
// Decoding from host memory with the copies overlapped (two chunk buffers).
// ---------------------------------------------------------------------------
namespace {

struct HostLayout {
  size_t llr[2], hard[2], iters[2], ws[2], total;
};

size_t round256(size_t n) { return (n + 255) & ~static_cast<size_t>(255); }

HostLayout host_layout(const cbp_code* c, int chunk, size_t ws_bytes) {
  HostLayout L{};
  const size_t words = (static_cast<size_t>(c->N) + 31) / 32;
  size_t off = 0;
  for (int b = 0; b < 2; ++b) {
    L.llr[b] = off;
    off += round256(static_cast<size_t>(chunk) * c->N * sizeof(float));
  }
  for (int b = 0; b < 2; ++b) {
    L.hard[b] = off;
    off += round256(static_cast<size_t>(chunk) * words * sizeof(uint32_t));
  }
  for (int b = 0; b < 2; ++b) {
    L.iters[b] = off;
    off += round256(static_cast<size_t>(chunk) * sizeof(int32_t));
  }
  for (int b = 0; b < 2; ++b) {  // chunks i and i + 1 may decode at the same time
    L.ws[b] = off;
    off += round256(ws_bytes);
  }
  L.total = off;
  return L;
}

int host_setup(const cbp_code* c, int chunk, const cbp_opts_t* opts, int* alg, float* alpha,
               int* stop, DeviceInfo** dio, Plan* pl, HostLayout* L) {
  if (!c || chunk < 1) return CBP_EINVAL;
  float* soft = nullptr;
  if (int rc = check_opts(opts, alg, alpha, stop, &soft)) return rc;
  if (soft) return CBP_EINVAL;
  int dev = 0;
  if (int rc = current_device(dio, &dev)) return rc;
  if (dev != c->dev) return CBP_EDEVICE;
  if (int rc = make_plan(c, **dio, *alg, chunk, pl, *stop)) return rc;
  *L = host_layout(c, chunk, pl->ws_bytes);
  return CBP_OK;
}

}  // namespace

int cbp_host_buffer_bytes(const cbp_code_t* c, int chunk, const cbp_opts_t* opts,
                          size_t* bytes) {
  if (!bytes) return CBP_EINVAL;
  int alg, stop;
  float alpha;
  DeviceInfo* di = nullptr;
  Plan pl;
  HostLayout L;
  if (int rc = host_setup(c, chunk, opts, &alg, &alpha, &stop, &di, &pl, &L)) return rc;
  *bytes = L.total;
  return CBP_OK;
}

int cbp_decode_host(const cbp_code_t* c, const float* llr_host, uint32_t* hard_host,
                    int32_t* iters_host, int max_iter, int batch, int chunk, void* dev_buf,
                    size_t dev_bytes, cbp_stream_t stream, const cbp_opts_t* opts) {
  if (!c || max_iter < 1 || batch < 0) return CBP_EINVAL;
  int alg, stop;
  float alpha;
  DeviceInfo* di = nullptr;
  Plan pl;
  HostLayout L;
  if (int rc = host_setup(c, chunk, opts, &alg, &alpha, &stop, &di, &pl, &L)) return rc;
  if (batch == 0) return CBP_OK;
  if (!llr_host || !hard_host || !iters_host || !dev_buf || !aligned(dev_buf, 256))
    return CBP_EINVAL;
  if (dev_bytes < L.total) return CBP_EWORKSPACE;
  unsigned char* base = static_cast<unsigned char*>(dev_buf);
  const cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  const size_t words = (static_cast<size_t>(c->N) + 31) / 32;
  const int n_chunks = static_cast<int>((static_cast<long long>(batch) + chunk - 1) / chunk);
  // chunks decode alternately on `stream` and on ks, each with its own workspace, so
  // that the CTAs of chunk i + 1 take the SMs that chunk i's tail leaves idle; cs copies
  cudaStream_t cs = nullptr, ks = nullptr;
  cudaEvent_t ev_in[2] = {nullptr, nullptr}, ev_dec[2] = {nullptr, nullptr}, ev_done = nullptr;
  int rc = CBP_OK;
  auto ok = [&](cudaError_t e) {
    if (e != cudaSuccess && rc == CBP_OK) rc = CBP_ECUDA;
    return rc == CBP_OK;
  };
  auto frames = [&](int i) { return std::min(chunk, batch - i * chunk); };
  auto h2d = [&](int i) {
    const int b = i & 1;
    return ok(cudaMemcpyAsync(base + L.llr[b], llr_host + static_cast<size_t>(i) * chunk * c->N,
                              static_cast<size_t>(frames(i)) * c->N * sizeof(float),
                              cudaMemcpyHostToDevice, cs)) &&
           ok(cudaEventRecord(ev_in[b], cs));
  };
  if (ok(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking)) &&
      ok(cudaStreamCreateWithFlags(&ks, cudaStreamNonBlocking)) &&
      ok(cudaEventCreateWithFlags(&ev_in[0], cudaEventDisableTiming)) &&
      ok(cudaEventCreateWithFlags(&ev_in[1], cudaEventDisableTiming)) &&
      ok(cudaEventCreateWithFlags(&ev_dec[0], cudaEventDisableTiming)) &&
      ok(cudaEventCreateWithFlags(&ev_dec[1], cudaEventDisableTiming)) &&
      ok(cudaEventCreateWithFlags(&ev_done, cudaEventDisableTiming))) {
    // the copy and decode streams start after the work the caller queued on `stream`
    ok(cudaEventRecord(ev_done, st)) && ok(cudaStreamWaitEvent(cs, ev_done, 0)) &&
        ok(cudaStreamWaitEvent(ks, ev_done, 0));
    for (int i = 0; i < std::min(2, n_chunks) && rc == CBP_OK; ++i) h2d(i);
    for (int i = 0; i < n_chunks && rc == CBP_OK; ++i) {
      const int b = i & 1, n = frames(i);
      KParams p = code_params(c, *di, pl, n, max_iter, stop, alpha);
      p.llr = reinterpret_cast<const float*>(base + L.llr[b]);
      p.hard = reinterpret_cast<uint32_t*>(base + L.hard[b]);
      p.iters = reinterpret_cast<int32_t*>(base + L.iters[b]);
      p.ws = reinterpret_cast<float*>(base + L.ws[b]);
      const cudaStream_t kst = b ? ks : st;
      if (!ok(cudaStreamWaitEvent(kst, ev_in[b], 0)) ||
          !ok(launch_decoder(pl.v, p, pl.grid, pl.threads, pl.smem, kst)) ||
          !ok(cudaEventRecord(ev_dec[b], kst)) || !ok(cudaStreamWaitEvent(cs, ev_dec[b], 0)) ||
          !ok(cudaMemcpyAsync(hard_host + static_cast<size_t>(i) * chunk * words,
                              base + L.hard[b], static_cast<size_t>(n) * words * sizeof(uint32_t),
                              cudaMemcpyDeviceToHost, cs)) ||
          !ok(cudaMemcpyAsync(iters_host + static_cast<size_t>(i) * chunk, base + L.iters[b],
                              static_cast<size_t>(n) * sizeof(int32_t), cudaMemcpyDeviceToHost,
                              cs)))
        break;
      // buffer b is free again once chunk i is decoded and its results copied out
      if (i + 2 < n_chunks) h2d(i + 2);
    }
    // `stream` completes after the last copy (which follows every decode)
    if (rc == CBP_OK) ok(cudaEventRecord(ev_done, cs)) && ok(cudaStreamWaitEvent(st, ev_done, 0));
  }
  // released once the queued work has finished
  for (cudaEvent_t e : {ev_in[0], ev_in[1], ev_dec[0], ev_dec[1], ev_done})
    if (e) cudaEventDestroy(e);
  if (cs) cudaStreamDestroy(cs);
  if (ks) cudaStreamDestroy(ks);
  return rc;
}

// ---------------------------------------------------------------------------
// Weighted CBP (differentiable decoder)
// ---------------------------------------------------------------------------
namespace {

int grad_setup(const cbp_code_t* c, int batch, int T, int ckpt, GParams* p, int* grid,
               int* threads, size_t* smem, size_t* ws_bytes, DeviceInfo** dio) {
  if (!c || batch < 0 || T < 1 || ckpt < 1 || ckpt > T) return CBP_EINVAL;
  if (c->Z > 512) return CBP_EUNSUPPORTED;
  DeviceInfo* di = nullptr;
  int dev = 0;
  if (int rc = current_device(&di, &dev)) return rc;
  if (dev != c->dev) return CBP_EDEVICE;
  const size_t ff = grad_frame_floats(c->N, c->M, c->E, T, ckpt);
  *ws_bytes = ff * sizeof(float) * static_cast<size_t>(batch);
  const size_t sm = sizeof(float4) * kPhiSegments + sizeof(BaseEdge) * c->nnzb +
                    sizeof(int) * ((c->mb + 1 + 3) & ~3) + sizeof(uint2) * ((c->nb + 1) & ~1) +
                    2 * sizeof(float) * static_cast<size_t>(T) * c->mb;  // gradients, weights
  if (sm > static_cast<size_t>(di->smem_optin)) return CBP_EUNSUPPORTED;
  const int F = std::max(1, 256 / c->Z);
  *threads = (F * c->Z + 31) / 32 * 32;
  *grid = static_cast<int>((static_cast<long long>(batch) + F - 1) / F);
  *smem = sm;
  GParams q{};
  q.status = c->d.status;
  q.edges = c->d.edges;
  q.rptr = c->d.rptr;
  q.cols = c->d.cols;
  q.cptr = c->d.cptr;
  q.phi_tab = di->tab;
  q.phi_xlo = di->xlo;
  q.Z = c->Z;
  q.mb = c->mb;
  q.nb = c->nb;
  q.nnzb = c->nnzb;
  q.N = c->N;
  q.M = c->M;
  q.E = c->E;
  q.batch = batch;
  q.T = T;
  q.ckpt = ckpt;
  q.nseg = (T + ckpt - 1) / ckpt;
  q.F = F;
  q.frame_floats = static_cast<long long>(ff);
  q.st_floats = static_cast<long long>((2 * static_cast<size_t>(c->N) + c->M + c->E + 3) &
                                       ~static_cast<size_t>(3));
  // the backward keeps the check-belief adjoints in shared memory when they fit
  const size_t gsb = sizeof(float) * static_cast<size_t>(F) * c->M;
  q.gs_shared = sm + gsb <= static_cast<size_t>(di->smem_optin) ? 1 : 0;
  q.gs_bytes = q.gs_shared ? static_cast<int>(gsb) : 0;
  *p = q;
  if (dio) *dio = di;
  return CBP_OK;
}

}  // namespace

int cbp_grad_workspace_bytes(const cbp_code_t* c, int batch, int T, int ckpt_every,
                             size_t* bytes) {
  if (!bytes) return CBP_EINVAL;
  GParams p;
  int grid, threads;
  size_t smem;
  return grad_setup(c, batch, T, ckpt_every, &p, &grid, &threads, &smem, bytes, nullptr);
}

int cbp_decode_weighted(const cbp_code_t* c, const float* llr, const float* weights, int T,
                        int ckpt_every, int batch, float* soft_out, void* workspace,
                        size_t workspace_bytes, cbp_stream_t stream) {
  GParams p;
  int grid, threads;
  size_t smem, need;
  if (int rc = grad_setup(c, batch, T, ckpt_every, &p, &grid, &threads, &smem, &need, nullptr))
    return rc;
  if (batch == 0) return CBP_OK;
  if (!llr || !weights || !soft_out || !workspace) return CBP_EINVAL;
  if (!aligned(llr, 4) || !aligned(weights, 4) || !aligned(soft_out, 4) || !aligned(workspace, 256))
    return CBP_EINVAL;
  if (workspace_bytes < need) return CBP_EWORKSPACE;
  p.llr = llr;
  p.w = weights;
  p.soft = soft_out;
  p.ws = static_cast<float*>(workspace);
  return launch_weighted_forward(p, grid, threads, smem, reinterpret_cast<cudaStream_t>(stream)) ==
                 cudaSuccess
             ? CBP_OK
             : CBP_ECUDA;
}

int cbp_decode_grad(const cbp_code_t* c, const float* llr, const float* weights, int T,
                    int ckpt_every, int batch, const float* grad_soft, float* grad_weights,
                    float* grad_llr, void* workspace, size_t workspace_bytes,
                    cbp_stream_t stream) {
  GParams p;
  int grid, threads;
  size_t smem, need;
  if (int rc = grad_setup(c, batch, T, ckpt_every, &p, &grid, &threads, &smem, &need, nullptr))
    return rc;
  if (!grad_weights || !aligned(grad_weights, 4)) return CBP_EINVAL;
  const cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  if (cudaMemsetAsync(grad_weights, 0, sizeof(float) * static_cast<size_t>(T) * c->mb, st) !=
      cudaSuccess)
    return CBP_ECUDA;
  if (batch == 0) return CBP_OK;
  if (!llr || !weights || !grad_soft || !workspace) return CBP_EINVAL;
  if (!aligned(llr, 4) || !aligned(weights, 4) || !aligned(grad_soft, 4) ||
      !aligned(workspace, 256) || (grad_llr && !aligned(grad_llr, 4)))
    return CBP_EINVAL;
  if (workspace_bytes < need) return CBP_EWORKSPACE;
  p.llr = llr;
  p.w = weights;
  p.gsoft = grad_soft;
  p.gw = grad_weights;
  p.gllr = grad_llr;
  p.ws = static_cast<float*>(workspace);
  return launch_weighted_backward(p, grid, threads, smem, st) == cudaSuccess ? CBP_OK : CBP_ECUDA;
}

// ---------------------------------------------------------------------------
// cbp_decode_noalloc: the decoder scratch in a fixed device array of this file.
// Host code never dereferences g_noalloc_scratch (its name is a host-side stand-in);
// the device address is looked up once per device and passed to the kernel.
// ---------------------------------------------------------------------------
static __device__ __align__(256) unsigned char g_noalloc_scratch[CBP_NOALLOC_SCRATCH_BYTES];

namespace {
void* g_noalloc_ptr[kMaxDevices] = {};

int noalloc_scratch(int dev, void** out) {
  std::lock_guard<std::mutex> lk(g_mu);
  if (!g_noalloc_ptr[dev]) {
    void* ptr = nullptr;
    if (cudaGetSymbolAddress(&ptr, g_noalloc_scratch) != cudaSuccess || !ptr) return CBP_ECUDA;
    g_noalloc_ptr[dev] = ptr;
  }
  *out = g_noalloc_ptr[dev];
  return CBP_OK;
}
}  // namespace

int cbp_decode_noalloc(const cbp_code_t* c, const float* llr, uint32_t* hard_out,
                       int32_t* iters_out, int max_iter, int batch, cbp_stream_t stream) {
  if (!c || max_iter < 1 || batch < 0) return CBP_EINVAL;
  if (batch == 0) return CBP_OK;
  if (!llr || !hard_out || !iters_out) return CBP_EINVAL;
  if (!aligned(llr, 16) || !aligned(hard_out, 4) || !aligned(iters_out, 4)) return CBP_EINVAL;
  DeviceInfo* di = nullptr;
  int dev = 0;
  if (int rc = current_device(&di, &dev)) return rc;
  if (dev != c->dev) return CBP_EDEVICE;
  void* scratch = nullptr;
  if (int rc = noalloc_scratch(dev, &scratch)) return rc;
  Plan pl;
  if (int rc = make_plan(c, *di, ALG_CBP_SP, batch, &pl, CBP_STOP_SYNDROME, false)) return rc;
  // Fit the launch into the array: fewer CTAs, and if one CTA is still too big, fewer
  // frame slots per CTA.  Slots loop over frames, so any grid decodes the whole batch.
  const size_t cap = CBP_NOALLOC_SCRATCH_BYTES;
  const size_t slot_bytes = static_cast<size_t>(pl.ws.slot) * sizeof(float);
  if (slot_bytes > cap) return CBP_EWORKSPACE;
  if (static_cast<size_t>(pl.F) * slot_bytes > cap) {
    pl.F = static_cast<int>(cap / slot_bytes);
    pl.threads = (pl.F * c->Z + 31) / 32 * 32;
    pl.smem = shared_fixed_bytes(pl.v, c->shape(), pl.F) +
              static_cast<size_t>(pl.F) * pl.sh_frame * sizeof(float);
  }
  const long long max_grid = static_cast<long long>(cap / (pl.F * slot_bytes));
  pl.grid = static_cast<int>(std::min<long long>(pl.grid, max_grid));
  pl.ws_bytes = static_cast<size_t>(pl.grid) * pl.F * slot_bytes;

  KParams p = code_params(c, *di, pl, batch, max_iter, CBP_STOP_SYNDROME, 0.75f);
  p.llr = llr;
  p.hard = hard_out;
  p.iters = iters_out;
  p.ws = static_cast<float*>(scratch);
  cudaError_t e = launch_decoder(pl.v, p, pl.grid, pl.threads, pl.smem,
                                 reinterpret_cast<cudaStream_t>(stream));
  return e == cudaSuccess ? CBP_OK : CBP_ECUDA;
}

// ---------------------------------------------------------------------------
// Several codes in one persistent launch (CBP-SP).
// ---------------------------------------------------------------------------
}  // extern "C"

namespace {

struct MultiPlan {
  MultiParams mp{};
  int grid = 0, threads = 0, ctas_per_sm = 0, chunks = 0, fpt = 1;
  bool chk = false, self_last = false;
  size_t smem = 0, ws_bytes = 0;
};

constexpr size_t kCounterBytes = 256;  // work counter at the start of the workspace
constexpr int kDefaultTailPercent = 20;  // cbp_multi_opts_t::tail_percent == 0

// Lane groups, shared memory and workspace of every item under one CTA shape, and the
// work list: each item's main segment (chunks of `rounds` frame rounds), heaviest chunk
// first (a chunk's time grows with the code's base entries and with the frame rounds it
// holds), then the items' tail segments in the same order: the last tail_pct percent of
// each item's frames in chunks of one round, so that the launch ends on short chunks.
int multi_plan_try(const cbp_multi_item_t* items, int n, int max_iter, int stop, bool chk,
                   int fpt, int threads, int ctas_target, int rounds, int tail_pct,
                   MultiPlan* out) {
  DeviceInfo* di = nullptr;
  int dev = 0;
  if (int rc = current_device(&di, &dev)) return rc;
  // the weight-1-last instance serves a launch whose codes all qualify
  bool self_last = fpt == 1;
  for (int i = 0; i < n; ++i)
    if (items[i].batch > 0 && !items[i].code->self_last) self_last = false;
  void* kern = sp_multi_kernel_ptr(chk, fpt, self_last);
  cudaFuncAttributes fa;
  if (cudaFuncGetAttributes(&fa, kern) != cudaSuccess) return CBP_ECUDA;
  if (threads > fa.maxThreadsPerBlock) return CBP_EINVAL;
  const long long stat = static_cast<long long>(fa.sharedSizeBytes);
  const long long budget_sm = di->smem_sm / ctas_target - 1024 - stat;
  const long long budget = std::min<long long>(budget_sm, di->smem_optin - stat);
  MultiPlan pl;
  pl.threads = threads;
  pl.fpt = fpt;
  pl.chk = chk;
  pl.self_last = self_last;
  const Variant v{ALG_CBP_SP, chk, fpt};
  std::vector<int> order;
  std::vector<KParams> kp(n);
  std::vector<int> cf(n, 0), cf1(n, 0);
  long long ws_cta = 0;
  for (int i = 0; i < n; ++i) {
    const cbp_code* c = items[i].code;
    if (c->dev != dev) return CBP_EDEVICE;
    if (c->Z > threads) return CBP_EUNSUPPORTED;
    if (items[i].batch == 0) continue;
    const Shape sh = c->shape();
    const size_t fr = shared_frame_floats(v, sh);
    int G = 0;
    size_t smem = 0;
    for (int g = 1; g * c->Z <= threads; ++g) {
      const size_t b = shared_fixed_bytes(v, sh, g) + g * fr * sizeof(float);
      if (static_cast<long long>(b) > budget) break;
      G = g;
      smem = b;
    }
    if (G == 0) return CBP_EUNSUPPORTED;
    Plan cp;
    cp.v = v;
    cp.F = G;
    cp.grid = 0;
    cp.ws = ws_layout(v, sh);
    cp.sh_frame = static_cast<int>(fr);
    kp[i] = code_params(c, *di, cp, items[i].batch, max_iter, stop, 0.75f);
    kp[i].llr = items[i].llr;
    kp[i].hard = items[i].hard_out;
    kp[i].iters = items[i].iters_out;
    cf[i] = G * fpt * rounds;
    cf1[i] = G * fpt;
    pl.smem = std::max(pl.smem, smem);
    ws_cta = std::max<long long>(ws_cta, static_cast<long long>(G) * cp.ws.slot);
    order.push_back(i);
  }
  std::stable_sort(order.begin(), order.end(), [&](int a, int b) {
    return 1LL * items[a].code->nnzb * rounds > 1LL * items[b].code->nnzb * rounds;
  });
  pl.mp.ncodes = static_cast<int>(order.size());
  std::vector<int> split(n, 0);  // first frame of the item's tail segment
  for (size_t j = 0; j < order.size(); ++j) {
    const int i = order[j], b = items[i].batch;
    kp[i].ws_cta = ws_cta;
    pl.mp.code[j] = kp[i];
    long long tail = (1LL * b * tail_pct + 99) / 100;
    tail = std::min<long long>(b, (tail + cf1[i] - 1) / cf1[i] * cf1[i]);
    split[i] = b - static_cast<int>(tail);
  }
  long long chunks = 0;
  int ns = 0;
  auto add_seg = [&](int j, int f0, int f1, int frames) {
    if (f1 <= f0) return true;
    chunks += (f1 - f0 + frames - 1) / frames;
    if (chunks > (1LL << 30)) return false;
    pl.mp.seg_code[ns] = j;
    pl.mp.seg_frame0[ns] = f0;
    pl.mp.seg_frame1[ns] = f1;
    pl.mp.seg_frames[ns] = frames;
    pl.mp.seg_end[ns] = static_cast<int>(chunks);
    ++ns;
    return true;
  };
  for (size_t j = 0; j < order.size(); ++j)
    if (!add_seg(static_cast<int>(j), 0, split[order[j]], cf[order[j]])) return CBP_EUNSUPPORTED;
  for (size_t j = 0; j < order.size(); ++j)
    if (!add_seg(static_cast<int>(j), split[order[j]], items[order[j]].batch, cf1[order[j]]))
      return CBP_EUNSUPPORTED;
  pl.mp.nseg = ns;
  pl.chunks = static_cast<int>(chunks);
  int ctas = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&ctas, kern, threads, pl.smem) != cudaSuccess)
    return CBP_ECUDA;
  if (ctas < 1) return CBP_EUNSUPPORTED;
  pl.ctas_per_sm = ctas;
  pl.grid = static_cast<int>(std::max(1LL, std::min<long long>(chunks, 1LL * di->sms * ctas)));
  pl.ws_bytes = kCounterBytes + static_cast<size_t>(pl.grid) * ws_cta * sizeof(float);
  *out = pl;
  return CBP_OK;
}

int multi_plan(const cbp_multi_item_t* items, int n, const cbp_multi_opts_t* o, int max_iter,
               MultiPlan* out) {
  if (n < 0 || (n > 0 && !items)) return CBP_EINVAL;
  if (n > CBP_MULTI_MAX_ITEMS) return CBP_EINVAL;
  cbp_multi_opts_t d{};
  d.chk_shared = -1;
  if (o) d = *o;
  const int fpt = d.frames_per_group == 0 ? 1 : d.frames_per_group;
  if (fpt != 1 && fpt != 2) return CBP_EINVAL;
  const int tmax = fpt == 2 ? 384 : 768;
  const int threads = d.threads == 0 ? tmax : d.threads;
  if (threads < 32 || threads > tmax || threads % 32) return CBP_EINVAL;
  const int ctas = d.ctas_per_sm == 0 ? 1 : d.ctas_per_sm;
  const int rounds = d.rounds_per_chunk == 0 ? 4 : d.rounds_per_chunk;
  if (ctas < 1 || ctas > 32 || rounds < 1 || rounds > 4096) return CBP_EINVAL;
  if (d.stop_mode != CBP_STOP_SYNDROME && d.stop_mode != CBP_STOP_NONE) return CBP_EINVAL;
  if (d.tail_percent < -1 || d.tail_percent > 100) return CBP_EINVAL;
  const int tail = d.tail_percent == 0 ? kDefaultTailPercent : std::max(0, d.tail_percent);
  for (int i = 0; i < n; ++i)
    if (!items[i].code || items[i].batch < 0) return CBP_EINVAL;
  if (d.chk_shared == 0 || d.chk_shared == 1)
    return multi_plan_try(items, n, max_iter, d.stop_mode, d.chk_shared == 1, fpt, threads, ctas,
                          rounds, tail, out);
  const int rc = multi_plan_try(items, n, max_iter, d.stop_mode, true, fpt, threads, ctas, rounds,
                                tail, out);
  if (rc != CBP_EUNSUPPORTED) return rc;
  return multi_plan_try(items, n, max_iter, d.stop_mode, false, fpt, threads, ctas, rounds, tail,
                        out);
}

}  // namespace

extern "C" {

int cbp_multi_workspace_bytes(const cbp_multi_item_t* items, int n_items,
                              const cbp_multi_opts_t* opts, size_t* bytes) {
  if (!bytes) return CBP_EINVAL;
  MultiPlan pl;
  if (int rc = multi_plan(items, n_items, opts, 1, &pl)) return rc;
  *bytes = pl.mp.ncodes == 0 ? 0 : pl.ws_bytes;
  return CBP_OK;
}

int cbp_multi_launch_info(const cbp_multi_item_t* items, int n_items,
                          const cbp_multi_opts_t* opts, int* info) {
  if (!info) return CBP_EINVAL;
  MultiPlan pl;
  if (int rc = multi_plan(items, n_items, opts, 1, &pl)) return rc;
  info[0] = pl.mp.ncodes == 0 ? 0 : pl.grid;
  info[1] = pl.threads;
  info[2] = static_cast<int>(pl.smem);
  info[3] = pl.ctas_per_sm;
  info[4] = pl.chunks;
  info[5] = pl.chk ? 1 : 0;
  info[6] = pl.fpt;
  info[7] = pl.self_last ? 1 : 0;
  return CBP_OK;
}

int cbp_decode_multi(const cbp_multi_item_t* items, int n_items, int max_iter, void* workspace,
                     size_t workspace_bytes, cbp_stream_t stream, const cbp_multi_opts_t* opts) {
  if (max_iter < 1) return CBP_EINVAL;
  for (int i = 0; i < n_items && items; ++i) {
    const cbp_multi_item_t& it = items[i];
    if (it.batch <= 0) continue;
    if (!it.llr || !it.hard_out || !it.iters_out) return CBP_EINVAL;
    if (!aligned(it.llr, 16) || !aligned(it.hard_out, 4) || !aligned(it.iters_out, 4))
      return CBP_EINVAL;
  }
  MultiPlan pl;
  if (int rc = multi_plan(items, n_items, opts, max_iter, &pl)) return rc;
  if (pl.mp.ncodes == 0) return CBP_OK;
  if (!workspace || !aligned(workspace, 256)) return CBP_EINVAL;
  if (workspace_bytes < pl.ws_bytes) return CBP_EWORKSPACE;
  unsigned char* ws = static_cast<unsigned char*>(workspace);
  pl.mp.counter = reinterpret_cast<int*>(ws);
  for (int j = 0; j < pl.mp.ncodes; ++j)
    pl.mp.code[j].ws = reinterpret_cast<float*>(ws + kCounterBytes);
  const cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  if (cudaMemsetAsync(pl.mp.counter, 0, sizeof(int), st) != cudaSuccess) return CBP_ECUDA;
  return launch_multi(pl.chk, pl.fpt, pl.self_last, pl.mp, pl.grid, pl.threads, pl.smem, st) ==
                 cudaSuccess
             ? CBP_OK
             : CBP_ECUDA;
}

namespace {
int phi_call(const float* x, float* y, int64_t n, cbp_stream_t stream, bool deriv) {
  if (n < 0) return CBP_EINVAL;
  if (n == 0) return CBP_OK;
  if (!x || !y || !aligned(x, 4) || !aligned(y, 4)) return CBP_EINVAL;
  DeviceInfo* di = nullptr;
  if (int rc = current_device(&di, nullptr)) return rc;
  return launch_phi(x, y, n, di->tab, di->xlo, reinterpret_cast<cudaStream_t>(stream),
                    deriv) == cudaSuccess
             ? CBP_OK
             : CBP_ECUDA;
}
}  // namespace

int cbp_phi(const float* x, float* y, int64_t n, cbp_stream_t stream) {
  return phi_call(x, y, n, stream, false);
}

int cbp_phi_deriv(const float* x, float* y, int64_t n, cbp_stream_t stream) {
  return phi_call(x, y, n, stream, true);
}

int cbp_device_status(const cbp_code_t* c, cbp_stream_t stream, uint32_t* flags) {
  if (!c || !flags) return CBP_EINVAL;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return CBP_ECUDA;
  if (dev != c->dev) return CBP_EDEVICE;
  const cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  uint32_t v = 0;
  if (launch_status_take(c->d.status, st) != cudaSuccess ||
      cudaMemcpyAsync(&v, c->d.status + 1, sizeof v, cudaMemcpyDeviceToHost, st) !=
          cudaSuccess ||
      cudaStreamSynchronize(st) != cudaSuccess)
    return CBP_ECUDA;
  *flags = v;
  return CBP_OK;
}

int cbp_edge_ceiling(int ctas, int iters, float* sink, size_t sink_floats, cbp_stream_t stream,
                     int64_t* edge_updates, int* ctas_used) {
  if (iters < 1 || !sink || !edge_updates || !aligned(sink, 4)) return CBP_EINVAL;
  DeviceInfo* di = nullptr;
  if (int rc = current_device(&di, nullptr)) return rc;
  if (ctas <= 0) {
    int per_sm = 0;
    if (edge_ceiling_ctas_per_sm(&per_sm) || per_sm < 1) return CBP_ECUDA;
    ctas = per_sm * di->sms;
  }
  if (static_cast<size_t>(ctas) * 512 > sink_floats) return CBP_EINVAL;
  long long edges = 0;
  if (launch_edge_ceiling(di->tab, di->xlo, ctas, iters, sink,
                          reinterpret_cast<cudaStream_t>(stream), &edges) != cudaSuccess)
    return CBP_ECUDA;
  *edge_updates = edges;
  if (ctas_used) *ctas_used = ctas;
  return CBP_OK;
}

const char* cbp_strerror(int s) {
  switch (s) {
    case CBP_OK: return "success";
    case CBP_EINVAL: return "invalid argument";
    case CBP_ENOMEM: return "device allocation failed";
    case CBP_ECUDA: return "CUDA runtime or launch error";
    case CBP_EUNSUPPORTED: return "unsupported code size or option";
    case CBP_EWORKSPACE: return "workspace too small";
    case CBP_EDEVICE: return "code handle belongs to another device";
  }
  return "unknown status";
}

}  // extern "C"
