// Internal declarations shared by the libcbp translation units.
#pragma once

#include <cuda_runtime.h>

#include <cstddef>
#include <cstdint>

#include "cbp.h"

namespace cbp {

// ----------------------------------------------------------------------------
// phi(x) = -log tanh(x/2), Eq. (s2e5), in FP32.
// phi(clamp(x, X_LO, 30)) with X_LO = fl32(phi(30)); cubic Taylor polynomial around
// the nearest grid centre: below 2 the FP32 values whose low 18 mantissa bits are
// zero (bit patterns (2688 + i) << 18, i = 0..1408, i.e. 2^-43 .. 2.0), local variable
// t = (x - centre) / h with h = 2^e(centre); from 2 to 30 the centres k/16, h = 1/16.
// The coefficients are phi^(k)(m) h^k / k! rounded to FP32.  The device table holds
// them divided by h^k (exact: h is a power of two and no value leaves the normal FP32
// range), so the kernels evaluate the same Horner steps on d = x - centre (exact by
// Sterbenz) without forming t; every rounding is the scaled one times a power of two,
// so the result is bit-identical to the t form.
// ----------------------------------------------------------------------------
constexpr int kPhiLogBase = 2688;
constexpr int kPhiLogCount = 1409;
constexpr int kPhiSegments = kPhiLogCount + 449;

// Host: fill the coefficient table (4 floats per centre, the t form) and the lower clamp.
void phi_table_host(float* coef, float* xlo);
// Host: the device form of the table (coefficient k divided by h^k).
void phi_table_device_form(const float* coef, float* dev);

__device__ __forceinline__ float phi_eval(float x, float xlo, const float4* __restrict__ tab) {
  x = fminf(fmaxf(x, xlo), 30.0f);
  // below 2: nearest centre cb (round the low 18 mantissa bits), d = x - cb
  const uint32_t cb = (__float_as_uint(x) + 0x20000u) & 0xFFFC0000u;
  const float dl = __fsub_rn(x, __uint_as_float(cb));
  // 2 to 30: k = rint(16x) by adding 1.5 * 2^23 (16x is exact and below 2^22), d = x - k/16
  constexpr float kMagic = 12582912.0f;
  const float y = __fmaf_rn(x, 16.0f, kMagic);
  const float du = __fmaf_rn(__fsub_rn(y, kMagic), -0.0625f, x);
  const bool lo = x < 2.0f;
  const float d = lo ? dl : du;
  const int i = lo ? static_cast<int>(cb >> 18) - kPhiLogBase
                   : static_cast<int>(__float_as_uint(y) - __float_as_uint(kMagic)) +
                         (kPhiLogCount - 32);
  const float4 c = tab[i];
  float p = __fmaf_rn(c.w, d, c.z);
  p = __fmaf_rn(p, d, c.y);
  return __fmaf_rn(p, d, c.x);
}

// Derivative of phi_eval: the derivative of the centre's cubic, c1 + d (2 c2 + 3 c3 d),
// on the device form of the table; 0 where the clamp holds.
__device__ __forceinline__ float phi_deriv(float x, float xlo, const float4* __restrict__ tab) {
  const bool inside = x >= xlo && x <= 30.0f;
  x = fminf(fmaxf(x, xlo), 30.0f);
  const uint32_t cb = (__float_as_uint(x) + 0x20000u) & 0xFFFC0000u;
  const float dl = __fsub_rn(x, __uint_as_float(cb));
  constexpr float kMagic = 12582912.0f;
  const float y = __fmaf_rn(x, 16.0f, kMagic);
  const float du = __fmaf_rn(__fsub_rn(y, kMagic), -0.0625f, x);
  const bool lo = x < 2.0f;
  const float d = lo ? dl : du;
  const int i = lo ? static_cast<int>(cb >> 18) - kPhiLogBase
                   : static_cast<int>(__float_as_uint(y) - __float_as_uint(kMagic)) +
                         (kPhiLogCount - 32);
  const float4 c = tab[i];
  const float dp = __fmaf_rn(__fmaf_rn(3.0f * c.w, d, 2.0f * c.z), d, c.y);
  return inside ? dp : 0.0f;
}

// ----------------------------------------------------------------------------
// Code tables (built on the host by cbp_code_create).
// ----------------------------------------------------------------------------
// One entry per non-zero base entry, row-major, ascending column inside a row.
struct BaseEdge {
  uint16_t c;      // base column
  uint16_t s;      // shift
  uint16_t pr;     // predecessor row: the previous row (cyclically) holding column c
  uint16_t ps;     // shift of the predecessor entry
  uint16_t pe;     // index of the predecessor entry in this list
  uint16_t flags;  // kFirst: r is the first row of column c; kSelf: c has weight 1
  uint32_t pad;    // low 16 bits: index of column c among the columns of its kind
                   // (weight >= 2 columns, or weight-1 columns)
};
// kLast: r is the last row of column c (the check a flushed posterior reads).
constexpr uint16_t kFirst = 1, kSelf = 2, kLast = 16;

// Column-major view: the rows of column c in ascending order (flooding posterior).
struct ColEntry {
  uint16_t r, s, e, pad;
};

// The CBP-SP kernel's view of a base entry (row r, column c, shift s) for lane z, with
// lane-independent parts precomputed (Z is fixed per code).  With s' = 0 for a weight-1
// column (its state is indexed by the check lane) and s' = s otherwise, and
// d = (s - ps) mod Z for the predecessor entry (pr, ps, pe):
//   x = A | first << 30 | weight1 << 31, A = idx * Z + s'  (idx: compact column index)
//   y = pr * Z + d,  z = pe * Z + d,  w = (Z - s') | (Z - d) << 16
// so that, with u(T) = (z >= T ? Z : 0):  variable slot = A + z - u(Z - s'),
// predecessor check = y + z - u(Z - d),  predecessor R slot = z + z - u(Z - d).
using SpEdge = uint4;
constexpr uint32_t kSpFirst = 1u << 30, kSpSelf = 1u << 31, kSpMask = kSpFirst - 1;

// Device status word of a code handle (cbp_device_status): bits the kernels set instead of
// trapping when an input breaks the ABI's contract.
constexpr uint32_t kStatusNonFiniteLlr = 1u;  // a frame's channel LLRs hold NaN or +-Inf

__device__ __forceinline__ bool non_finite(float x) {
  return (__float_as_uint(x) & 0x7f800000u) == 0x7f800000u;
}

// Edge record of the wavefront-schedule kernel (cbp_level.cu), checks and edges in level
// order: x = v | kSpFirst (first check of v) | kSpSelf (v has one check), y = the
// predecessor check of v (cyclically), z = the predecessor's edge to v.
using LvlEdge = uint4;

struct CodeDev {
  uint32_t* status = nullptr;  // [2]: live flags, last value taken by cbp_device_status
  int* lvl_ptr = nullptr;      // [nlev + 1] wavefront schedule (null when not built)
  int* lvl_e0 = nullptr;       // [M + 1] first edge of each level-ordered check
  LvlEdge* lvl_edge = nullptr;  // [E]
  uint2* lvl_rec8 = nullptr;   // [E] 8-byte records (M <= 4096, E < 2^20), else null
  int* last_chk = nullptr;     // [N] the last check of each variable (level order)
  int* lvl_cptr = nullptr;     // [N + 1] each variable's edges ...
  int* lvl_cedge = nullptr;    // [E] ... by level-ordered index, ascending check index
  BaseEdge* edges = nullptr;  // [nnzb]
  SpEdge* spe = nullptr;      // [nnzb], CBP-SP kernel records
  int* rptr = nullptr;        // [mb + 1]
  ColEntry* cols = nullptr;   // [nnzb], column-major
  int* cptr = nullptr;        // [nb + 1]
};

// Kernel parameters (passed by value).
struct KParams {
  const float* llr;
  uint32_t* status;      // the code's device status word
  uint32_t* hard;
  int32_t* iters;
  float* soft;
  float* ws;
  const BaseEdge* edges;
  const SpEdge* spe;
  const int* rptr;
  const ColEntry* cols;
  const int* cptr;
  const float4* phi_tab;
  float phi_xlo;
  int Z, mb, nb, nnzb, N, M, E, words;
  int batch, max_iter, stop;
  float alpha;
  int F;                 // lane groups per CTA (each decodes fpt frames)
  int team_groups;       // lane groups per independently synchronised team (>= F: one team)
  int slots;             // frame slots of the launch: gridDim.x * F * fpt
  int maxdeg;
  int test_row;          // CBP-SP: base row whose checks are tested first at a sweep's end
  int ncomp, nself;      // columns of weight >= 2 / of weight 1
  long long ws_slot;     // floats of workspace per lane group
  long long ws_cta;      // CBP-SP: floats of workspace per CTA (>= F * ws_slot)
  long long ws_off_sv;   // offset (floats) of the weight-1 column state
  long long ws_off_s;    // CBP-SP: check-beliefs when not shared; min-sum: check state
  long long ws_off_c;    // CBP min-sum: (min1, min2) per check when not shared
  int sh_frame;          // floats of shared memory per lane group
  // frame-parallel CBP-SP (cbp_fp.cu): frame slots of the launch (one per thread) and the
  // offsets (floats) of SV, S, R and the decision bits in the workspace; QP is at 0
  long long fp_slots, fp_off_sv, fp_off_s, fp_off_r, fp_off_b;
  // wavefront-schedule CBP-SP (cbp_level.cu): the code's level tables, the number of
  // levels and the lanes of a group
  const int* lvl_ptr;
  const int* lvl_e0;
  const LvlEdge* lvl_edge;
  const uint2* lvl_rec8;
  const int* last_chk;
  const int* lvl_cptr;
  const int* lvl_cedge;
  int nlev, lvl_lanes;
  int lvl_test;           // the widest level (tested first at a sweep's end)
};

// Several codes in one launch (CBP-SP): per-code parameters and the chunk list.
// The work list is a sequence of segments; a segment is a frame range [frame0, frame1)
// of one code cut into chunks of `frames` frames.  Each code has a main segment and,
// optionally, a tail segment of one-round chunks placed after every main segment.
constexpr int kMaxMultiCodes = 8;
constexpr int kMaxMultiSegs = 2 * kMaxMultiCodes;
struct MultiParams {
  KParams code[kMaxMultiCodes];
  int seg_code[kMaxMultiSegs];    // index into code[]
  int seg_end[kMaxMultiSegs];     // exclusive prefix end of the segments' chunks
  int seg_frame0[kMaxMultiSegs];  // first frame of the segment
  int seg_frame1[kMaxMultiSegs];  // end of the segment's frames
  int seg_frames[kMaxMultiSegs];  // frames per chunk
  int nseg;
  int* counter;                      // next chunk (zeroed before the launch)
  int ncodes;
};

enum Alg { ALG_CBP_SP = 0, ALG_CBP_NMS = 1, ALG_LBP_NMS = 2, ALG_FBP_SP = 3 };

struct Variant {
  int alg;
  bool chk_shared;  // check state in shared memory (else in the workspace)
  int fpt = 1;      // frames per lane group (CBP-SP: 1 or 2, interleaved)
  bool wide = false;  // CBP-SP: instance that allows 1024 threads per CTA (Z > 512)
  bool win = false;   // CBP-SP with the paper-literal stop (CBP_STOP_WINDOW)
  bool self_last = false;  // CBP-SP, one frame per group: every weight-1 edge ends its row
  bool fp = false;         // CBP-SP, frame-parallel kernel: one frame per thread
  bool rstore = false;     // CBP min-sum: C2V messages kept per edge (no rebuild)
  bool lvl = false;        // CBP-SP / min-sum on the wavefront schedule of the expanded graph
  bool shrec = false;      // that kernel with its edge records in shared memory
  int deg = 0;             // wavefront flooding kernel: its degree bucket (8, 16 or 32)
};

// Sizes that fix the shared-memory and workspace layout of a launch.
struct Shape {
  int Z, N, M, E, nnzb, mb, nb, words, ncomp, nself;
};
size_t shared_fixed_bytes(const Variant& v, const Shape& s, int groups);
size_t shared_frame_floats(const Variant& v, const Shape& s);  // per lane group
// Workspace floats per lane group and the offsets of its parts (see KParams).
struct WsLayout {
  long long slot = 0, off_sv = 0, off_s = 0, off_c = 0;
};
WsLayout ws_layout(const Variant& v, const Shape& s);

// Launchers (cbp_dispatch.cu).
cudaError_t launch_decoder(const Variant& v, const KParams& p, int grid, int threads,
                           size_t smem, cudaStream_t st);
cudaError_t decoder_func_attrs(const Variant& v, cudaFuncAttributes* a);
cudaError_t decoder_set_smem(const Variant& v, int bytes);
cudaError_t decoder_occupancy(const Variant& v, int threads, size_t smem, int* ctas);
void* sp_kernel_ptr(bool chk_shared, int fpt, bool wide, bool self_last);  // cbp_sp.cu
void* level_kernel_ptr(bool shrec);  // cbp_level.cu
void* lbp_level_kernel_ptr(bool shv);
void* nms_level_kernel_ptr(bool shrec);
void* fbp_level_kernel_ptr(bool shv, int maxdeg);
int level_max_threads();
void* sp_multi_kernel_ptr(bool chk_shared, int fpt, bool self_last);  // cbp_sp.cu
void* sp_win_kernel_ptr(bool chk_shared);                   // cbp_sp.cu
cudaError_t launch_multi(bool chk_shared, int fpt, bool self_last, const MultiParams& mp, int grid,
                         int threads, size_t smem, cudaStream_t st);
void* minsum_kernel_ptr(int alg, bool chk_shared, bool rstore);  // cbp_minsum.cu
void* fp_kernel_ptr();                                       // cbp_fp.cu
int fp_threads();                                            // cbp_fp.cu: threads per CTA
void* flood_kernel_ptr();              // cbp_flood.cu
cudaError_t launch_phi(const float* x, float* y, long long n, const float4* tab, float xlo,
                       cudaStream_t st, bool deriv);
cudaError_t launch_status_take(uint32_t* status, cudaStream_t st);  // cbp_flood.cu
// CBP-SP edge-update ceiling (cbp_ceiling.cu): 512 threads per CTA.
cudaError_t launch_edge_ceiling(const float4* tab, float xlo, int blocks, int iters,
                                float* sink, cudaStream_t st, long long* edges);
int edge_ceiling_ctas_per_sm(int* ctas);

// Weighted CBP (differentiable decoder), cbp_grad.cu.
struct GParams {
  const float* llr;
  uint32_t* status;      // the code's device status word
  const float* w;        // [T][mb]
  float* soft;           // forward output [batch][N]
  const float* gsoft;    // backward input [batch][N]
  float* gw;             // [T][mb], accumulated
  float* gllr;           // [batch][N] or null
  float* ws;
  const BaseEdge* edges;
  const int* rptr;
  const ColEntry* cols;
  const int* cptr;
  const float4* phi_tab;
  float phi_xlo;
  int Z, mb, nb, nnzb, N, M, E;
  int batch, T, ckpt, nseg, F;
  long long frame_floats, st_floats;
  int gs_shared;         // backward: check-belief adjoints in shared memory (F * M floats)
  int gs_bytes;          // their bytes, added to the launch's dynamic shared memory
};
size_t grad_frame_floats(int N, int M, int E, int T, int ckpt);
cudaError_t launch_weighted_forward(const GParams& p, int grid, int threads, size_t smem,
                                    cudaStream_t st);
cudaError_t launch_weighted_backward(const GParams& p, int grid, int threads, size_t smem,
                                     cudaStream_t st);
cudaError_t grad_set_smem(int bytes);

constexpr int kMaxDeg = 32;     // row-degree limit of the two-pass (pooled) comparators
constexpr int kMaxDegCbpMs = 64;  // CBP min-sum: one sign bit per edge in a 64-bit mask

}  // namespace cbp
