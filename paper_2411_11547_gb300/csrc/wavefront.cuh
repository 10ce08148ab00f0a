// The Pair-HMM forward wavefront (Sec. III-B, redesigned for sm_103a).
//
// One pair is scored by a group of L lanes of a warp (G = 32/L pairs per warp).  Lane t
// owns K consecutive rows (read positions) of the DP matrices and keeps M, I, D of its rows
// in registers (Sec. III-B: full in-register recurrences).  At step s it computes column
// j = s - t of its rows; the values of the row just above its strip, at columns j and
// j-1, come from lane t-1 through __shfl_up_sync (Sec. III-B, Fig. 2), together with the
// haplotype code of the column.  Lane 0 reads 16 haplotype codes per 128-bit load.
//
// Emission (Eq. 4) is staged in shared memory as E[c][row] = beta * lambda for the six codes
// (A C G T N and "no column"), so one 128-bit load returns four rows' emissions for the
// column's code (Sec. III-B: the |Sigma| x m emission table).  With beta folded into E and
// alpha' = alpha/beta, Eq. 1 becomes M = E[h_j][i] * (alpha'_i M(i-1,j-1) + I(i-1,j-1) +
// D(i-1,j-1)): 3 FP32 pipe operations, plus 2 for Eq. 2 and 2 for Eq. 3, 7 per cell.
//
// Reads shorter than L*K are padded at the TOP: pad rows carry the row-0 boundary down
// unchanged (their I passes through with coefficient 1, their emissions are 0), so the last
// row of the last lane is always row m and the result is the running sum of its M + I
// (Sec. II-A result line).  The first real row takes I(0,j) = 0 through a zero I
// coefficient, and M(1,j) = lambda * beta * D(0,j-1) through the boundary value
// I + D = K0/n of the row above, which is the initialisation D(0,j) = 1/n times K0.
//
// Precision tiers (the FP64 rescue and per-lane exponents are not in the paper):
//   plain: one initial constant K0 (2^120 in FP32, 2^1020 in FP64), exact by linearity;
//   ext:   every 16 steps each lane renormalises its state by a power of two and tracks the
//          exponent; incoming boundary values are converted by 2^(E_up - E_own).  Exact up
//          to rounding because the recurrences are linear; never underflows.
#pragma once
#include <cmath>
#include <type_traits>
#include "phmm_internal.cuh"

namespace phmm {

template <typename T>
struct Num;

template <>
struct Num<float> {
  static constexpr float K0 = kK32;
  static constexpr int kMinExp = -126, kMaxExp = 127;
  __device__ __forceinline__ static int ilog2(float x) {
    return ((__float_as_int(x) >> 23) & 0xff) - 127;
  }
  __device__ __forceinline__ static float exp2i(int d) {
    if (d < kMinExp) return 0.f;
    if (d > kMaxExp) d = kMaxExp;
    return __int_as_float((d + 127) << 23);
  }
};

template <>
struct Num<double> {
  static constexpr double K0 = kK64;
  static constexpr int kMinExp = -1022, kMaxExp = 1023;
  __device__ __forceinline__ static int ilog2(double x) {
    return (int)((__double_as_longlong(x) >> 52) & 0x7ff) - 1023;
  }
  __device__ __forceinline__ static double exp2i(int d) {
    if (d < kMinExp) return 0.0;
    if (d > kMaxExp) d = kMaxExp;
    return __longlong_as_double((long long)(d + 1023) << 52);
  }
};

// Start of haplotype h inside the code buffer: 16-byte aligned (closed form, so no scan is
// needed).  Every haplotype has at least kHapGuard bytes of NULLC before its first code and
// after its last (the preparation kernel writes them), so a lane may read a window of codes
// that starts up to kHapGuard - 4 columns before column 1 or ends up to kHapGuard - 4 past
// column n without a bounds check.
constexpr int kHapGuard = 48;
__host__ __device__ __forceinline__ int64_t hap_start(int64_t hap_off_h, int64_t h) {
  return (hap_off_h + (2 * kHapGuard + 16) * h + kHapGuard + 15) & ~(int64_t)15;
}
// Bytes of the code buffer for haplotypes of sum_n bases in total.
__host__ __device__ __forceinline__ int64_t hap_code_bytes(int64_t sum_n, int64_t H) {
  return hap_start(sum_n, H) + 2 * kHapGuard;
}

// Shared-memory row stride (elements) of one lane's emission rows: a lane's 16-byte chunks
// must fall in distinct bank groups for 8 consecutive lanes, so the stride in 16-byte units
// is odd.
template <typename T, int K>
struct TableGeom {
  static constexpr int VW = 16 / sizeof(T);                  // elements per 128-bit load
  static constexpr int KV = (K + VW - 1) / VW * VW;          // rows rounded to whole vectors
  static constexpr int units = KV / VW;
  static constexpr int LS = (units % 2 == 1) ? KV : KV + VW;  // lane stride
  static constexpr int CS = 32 * LS;                         // code-plane stride
  static constexpr size_t warp_bytes = (size_t)kCodes * CS * sizeof(T);
};

template <typename T, int K>
__device__ __forceinline__ void store_vec(T *dst, const T *v);
template <>
__device__ __forceinline__ void store_vec<float, 4>(float *dst, const float *v) {
  *reinterpret_cast<float4 *>(dst) = make_float4(v[0], v[1], v[2], v[3]);
}
template <>
__device__ __forceinline__ void store_vec<double, 2>(double *dst, const double *v) {
  *reinterpret_cast<double2 *>(dst) = make_double2(v[0], v[1]);
}

// K rows of a lane's emission row: 128-bit loads.  The row is padded to whole vectors, so a
// partial last vector is read with one 128-bit load too (a 64-bit load at the odd 16-byte
// lane stride would put two lanes of a half-warp on the same bank).
template <typename T, int K>
__device__ __forceinline__ void load_rows(const T *src, T (&e)[K]) {
  constexpr int VW = 16 / sizeof(T);
#pragma unroll
  for (int r = 0; r < K; r += VW) {
    if constexpr (sizeof(T) == 4) {
      const float4 v = *reinterpret_cast<const float4 *>(src + r);
      e[r] = v.x;
      if (r + 1 < K) e[r + 1] = v.y;
      if (r + 2 < K) e[r + 2] = v.z;
      if (r + 3 < K) e[r + 3] = v.w;
    } else {
      const double2 v = *reinterpret_cast<const double2 *>(src + r);
      e[r] = v.x;
      if (r + 1 < K) e[r + 1] = v.y;
    }
  }
}

__device__ __forceinline__ double qual_at(const void *q, int f32, int64_t g) {
  return f32 ? (double)reinterpret_cast<const float *>(q)[g]
             : (double)reinterpret_cast<const uint8_t *>(q)[g];
}

// Row parameters of read position g: alpha' = alpha/beta, delta, zeta, Q.  be: the row's
// beta when the batch has a per-base gap-continuation track (FP64; the FP32 parameters were
// prepared with it), else 0 for the scalar beta.
template <typename T>
__device__ __forceinline__ void row_params(const FwdArgs &a, int64_t g, T &ap, T &dl, T &zt,
                                           T &Q, double be = 0.0) {
  if constexpr (sizeof(T) == 4) {
    RowParams v = a.rp[g];
    ap = v.x;
    dl = v.y;
    zt = v.z;
    Q = v.w;
  } else {
    const double bq = qual_at(a.bq, a.qual_f32, g), iq = qual_at(a.iq, a.qual_f32, g),
                 dq = qual_at(a.dq, a.qual_f32, g);
    Q = exp10(-bq / 10.0);
    dl = exp10(-iq / 10.0);
    zt = exp10(-dq / 10.0);
    const double al = a.alpha_mode ? 1.0 - exp10(-(iq + dq) / 10.0) : 1.0 - (dl + zt);
    ap = al / (be > 0.0 ? be : a.beta64);
  }
}

// Gap continuation of read position g for a plan with a per-base track: eps_i and
// beta_i = 1 - eps_i (FP32 from the prepared values, FP64 from the raw Phred value).
template <typename T>
__device__ __forceinline__ void row_gap(const FwdArgs &a, int64_t g, T &ep, T &be) {
  if constexpr (sizeof(T) == 4) {
    const float2 v = a.rgap[g];
    ep = v.x;
    be = v.y;
  } else {
    ep = exp10(-qual_at(a.gq, a.qual_f32, g) / 10.0);
    be = 1.0 - ep;
  }
}

// One column of a row tile's last row, handed to the next tile (E: the last lane's
// exponent, an exact small integer in T).
template <typename T>
struct alignas(16) TileCol {
  T M, I, X, E;
};

// Register state of one lane of the wavefront.
template <typename T, int K>
struct WfState {
  T M[K], I[K], D[K];  // the lane's rows at its current column
  T Md, Sd;            // row above the strip at the previous column: M and I + D
  T acc;               // running sum of M + I of the lane's last row
  T f;                 // 2^(E_up - E_own) (and the row bias) for values from the lane above
  int E;               // per-lane exponent (per-lane-exponent tier)
  int c;               // haplotype code of the lane's current column
};

// One wavefront step: lane t advances its K rows by one column (Eq. 1-3).
// `in3` receives the boundary values (M, I, D of the row above at this column, in the
// lane's own scale) for callers that record the step (the adjoint's recompute).
//
// PRIMED: the state holds D' = D / zeta instead of D (per row).  Eq. 3 becomes
// D'(i,j) = M(i,j-1) + eps D'(i,j-1), one FMA instead of a multiply and an FMA, and the
// I + D the next row needs is formed as I + zeta D' (an FMA instead of an add): 6 FP32
// operations per cell instead of 7.  The lane below receives I + D of the last row directly
// (in3[2] then holds I + D, not D).
// ABS_E: the table holds signed emissions (the sign marks a match, for the adjoint); the
// recurrence uses their magnitudes (a free operand modifier).
// TOP: lane 0 takes the row above its strip from (tM, tI, tT), already in its own scale,
// instead of the DP's row 0 (row tiles of long reads: the previous tile's last row).
// OWN: every lane passes the haplotype code of its own column in `cu` (no code exchange).
// GQ: a per-base gap-continuation track: row r's D chain takes er[r] instead of eps.
template <typename T, int L, int K, bool EXT, bool PRIMED = false, bool ABS_E = false,
          bool TOP = false, bool OWN = false, bool GQ = false>
__device__ __forceinline__ void wf_step(WfState<T, K> &st, int cu, int t, T bnd, T eps,
                                        const T *tbl, const T (&ap)[K], const T (&dl)[K],
                                        const T (&zt)[K], const T (&ei)[K], T (&in3)[3],
                                        T tM = 0, T tI = 0, T tT = 0, const T *er = nullptr) {
  constexpr unsigned FULL = 0xffffffffu;
  constexpr int CS = TableGeom<T, K>::CS;
  if constexpr (OWN) {
    st.c = cu;
  } else {
    const int cin = __shfl_up_sync(FULL, st.c, 1, L);
    st.c = (t == 0) ? cu : cin;
  }
  const T third = PRIMED ? st.I[K - 1] + zt[K - 1] * st.D[K - 1] : st.D[K - 1];
  T inM = __shfl_up_sync(FULL, st.M[K - 1], 1, L);
  T inI = __shfl_up_sync(FULL, st.I[K - 1], 1, L);
  T inD = __shfl_up_sync(FULL, third, 1, L);
  if (t == 0) {  // row 0 (or the last pad row): M = 0, I + D = K0 * D(0, j) carried in I
    if constexpr (TOP) {
      inM = tM;
      inI = tI;
      inD = tT;
    } else {
      inM = 0;
      inI = bnd;
      inD = PRIMED ? bnd : (T)0;
    }
  }
  if constexpr (EXT) {
    const T fe = (TOP && t == 0) ? (T)1 : st.f;
    inM *= fe;
    inI *= fe;
    inD *= fe;
  }
  in3[0] = inM;
  in3[1] = inI;
  in3[2] = inD;
  T e[K];
  load_rows<T, K>(tbl + st.c * CS, e);
#pragma unroll
  for (int r = K - 1; r >= 0; --r) {
    const T md = r ? st.M[r - 1] : st.Md;
    T sd;
    const T epr = GQ ? er[r] : eps;
    if constexpr (PRIMED) {
      sd = r ? st.I[r - 1] + zt[r - 1] * st.D[r - 1] : st.Sd;
      st.D[r] = st.M[r] + epr * st.D[r];            // Eq. 3 over zeta
    } else {
      sd = r ? st.I[r - 1] + st.D[r - 1] : st.Sd;
      st.D[r] = zt[r] * st.M[r] + epr * st.D[r];    // Eq. 3 (same row, previous column)
    }
    const T er = ABS_E ? fabs(e[r]) : e[r];
    st.M[r] = er * (ap[r] * md + sd);               // Eq. 1 (previous row, previous column)
  }
  st.I[0] = dl[0] * inM + ei[0] * inI;  // Eq. 2 (previous row, same column)
#pragma unroll
  for (int r = 1; r < K; ++r) st.I[r] = dl[r] * st.M[r - 1] + ei[r] * st.I[r - 1];
  st.Md = inM;
  st.Sd = PRIMED ? inD : inI + inD;
  st.acc += st.M[K - 1] + st.I[K - 1];
}

// Per-lane renormalisation by a power of two (exact).  A lane that holds only zeros (the
// wavefront has not reached it) takes the exponent that makes the next values from the lane
// above arrive near 1.  Returns whether the lane's state is nonzero.
template <typename T, int L, int K, int kBias>
__device__ __forceinline__ bool wf_rescale(WfState<T, K> &st, int t) {
  constexpr unsigned FULL = 0xffffffffu;
  T mx = st.Md > st.Sd ? st.Md : st.Sd;
#pragma unroll
  for (int r = 0; r < K; ++r) mx = fmax(mx, fmax(st.M[r], fmax(st.I[r], st.D[r])));
  if (t == L - 1) mx = fmax(mx, st.acc);
  const bool zero = !(mx > (T)0);
  if (!zero) {
    const int En = st.E + Num<T>::ilog2(mx);
    const T sc = Num<T>::exp2i(st.E - En);
#pragma unroll
    for (int r = 0; r < K; ++r) {
      st.M[r] *= sc;
      st.I[r] *= sc;
      st.D[r] *= sc;
    }
    st.Md *= sc;
    st.Sd *= sc;
    st.acc *= sc;
    st.E = En;
  }
  const T xb = fmax(st.M[K - 1], fmax(st.I[K - 1], st.D[K - 1]));
  const int Eup = __shfl_up_sync(FULL, st.E, 1, L);
  const T xbu = __shfl_up_sync(FULL, xb, 1, L);
  if (zero && t > 0)
    st.E = Eup - kBias * (K - 1) + (xbu > (T)0 ? Num<T>::ilog2(xbu) : 0);
  st.f = Num<T>::exp2i(t == 0 ? -st.E : Eup - st.E - kBias * (K - 1));
  return !zero;
}

// ---- packed FP32 path (fma.rn.f32x2 / mul.rn.f32x2: two lane operations per instruction,
// each rounded exactly as its scalar counterpart) --------------------------------------------
__device__ __forceinline__ unsigned long long pk2(float2 v) {
  unsigned long long r;
  asm("mov.b64 %0, {%1,%2};" : "=l"(r) : "f"(v.x), "f"(v.y));
  return r;
}
__device__ __forceinline__ float2 upk2(unsigned long long r) {
  float2 v;
  asm("mov.b64 {%0,%1}, %2;" : "=f"(v.x), "=f"(v.y) : "l"(r));
  return v;
}
__device__ __forceinline__ float2 ffma2(float2 a, float2 b, float2 c) {
  unsigned long long d;
  asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(pk2(a)), "l"(pk2(b)), "l"(pk2(c)));
  return upk2(d);
}
__device__ __forceinline__ float2 fmul2(float2 a, float2 b) {
  unsigned long long d;
  asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(pk2(a)), "l"(pk2(b)));
  return upk2(d);
}

// Lane state of the packed path: pair p holds rows p and p + K/2, so the row above a pair
// (rows p-1, p-1+K/2) is again one pair (for p = 0: the strip's input row and row K/2-1).
template <int K>
struct WfState2 {
  static constexpr int H = K / 2;
  float2 M[H], I[H], D[H];  // D holds D/zeta (Eq. 3 over zeta, as the PRIMED scalar step)
  float Md, Sd, acc, f;
  int E, c;
};

// The emission table of the packed path stores a lane's rows interleaved (p, p + K/2, p+1,
// ...): table position -> row.
template <int K>
__host__ __device__ constexpr int x2_row(int pos) {
  return (pos & 1) ? K / 2 + pos / 2 : pos / 2;
}

// One wavefront step of the packed path (extended-range FP32, D/zeta form; the same
// arithmetic as wf_step<float, L, K, true, true> per lane operation): 3.5 instructions per
// cell instead of 6; only the I chain down the rows (Eq. 2) stays scalar.
template <int L, int K, bool TOP = false, bool GQ = false>
__device__ __forceinline__ void wf_step_x2(WfState2<K> &st, int cu, int t, float bnd, float eps,
                                           const float *tbl, const float2 (&ap)[K / 2],
                                           const float2 (&dl)[K / 2], const float2 (&zt)[K / 2],
                                           const float2 (&ei)[K / 2], float tM = 0.f,
                                           float tI = 0.f, float tT = 0.f,
                                           const float2 *er2 = nullptr) {
  constexpr unsigned FULL = 0xffffffffu;
  constexpr int H = K / 2;
  constexpr int CS = TableGeom<float, K>::CS;
  const int cin = __shfl_up_sync(FULL, st.c, 1, L);
  st.c = (t == 0) ? cu : cin;
  const float third = fmaf(zt[H - 1].y, st.D[H - 1].y, st.I[H - 1].y);  // I + D of row K-1
  float inM = __shfl_up_sync(FULL, st.M[H - 1].y, 1, L);
  float inI = __shfl_up_sync(FULL, st.I[H - 1].y, 1, L);
  float inD = __shfl_up_sync(FULL, third, 1, L);
  if (t == 0) {
    if constexpr (TOP) {
      inM = tM;
      inI = tI;
      inD = tT;
    } else {
      inM = 0.f;
      inI = bnd;
      inD = bnd;
    }
  }
  const float fe = (TOP && t == 0) ? 1.f : st.f;
  inM *= fe;
  inI *= fe;
  inD *= fe;
  float e[K];
  load_rows<float, K>(tbl + st.c * CS, e);
  // I + D (= I + zeta D') of every row at the previous column, before the update
  float2 S[H];
#pragma unroll
  for (int p = 0; p < H; ++p) S[p] = ffma2(zt[p], st.D[p], st.I[p]);
  const float Mtop = st.M[H - 1].x, Stop = S[H - 1].x;  // row K/2-1, previous column
  const float2 eps2 = make_float2(eps, eps);
#pragma unroll
  for (int p = H - 1; p >= 0; --p) {
    const float2 md = p ? st.M[p - 1] : make_float2(st.Md, Mtop);
    const float2 sd = p ? S[p - 1] : make_float2(st.Sd, Stop);
    st.D[p] = ffma2(GQ ? er2[p] : eps2, st.D[p], st.M[p]);                 // Eq. 3 over zeta
    st.M[p] = fmul2(make_float2(e[2 * p], e[2 * p + 1]), ffma2(ap[p], md, sd));  // Eq. 1
  }
  // Eq. 2 down the rows: the products with the new M of the row above in pairs, the chain
  // through I scalar (rows 0 .. K/2-1, then K/2 .. K-1)
  float2 dM[H];
#pragma unroll
  for (int p = 0; p < H; ++p)
    dM[p] = fmul2(dl[p], p ? st.M[p - 1] : make_float2(inM, st.M[H - 1].x));
  float prev = inI;
#pragma unroll
  for (int p = 0; p < H; ++p) {
    st.I[p].x = fmaf(ei[p].x, prev, dM[p].x);
    prev = st.I[p].x;
  }
#pragma unroll
  for (int p = 0; p < H; ++p) {
    st.I[p].y = fmaf(ei[p].y, prev, dM[p].y);
    prev = st.I[p].y;
  }
  st.Md = inM;
  st.Sd = inD;
  st.acc += st.M[H - 1].y + st.I[H - 1].y;
}

// Per-lane renormalisation of the packed state (as wf_rescale).
template <int L, int K, int kBias>
__device__ __forceinline__ void wf_rescale_x2(WfState2<K> &st, int t) {
  constexpr unsigned FULL = 0xffffffffu;
  constexpr int H = K / 2;
  float mx = fmaxf(st.Md, st.Sd);
#pragma unroll
  for (int p = 0; p < H; ++p)
    mx = fmaxf(mx, fmaxf(fmaxf(fmaxf(st.M[p].x, st.M[p].y), fmaxf(st.I[p].x, st.I[p].y)),
                         fmaxf(st.D[p].x, st.D[p].y)));
  if (t == L - 1) mx = fmaxf(mx, st.acc);
  const bool zero = !(mx > 0.f);
  if (!zero) {
    const int En = st.E + Num<float>::ilog2(mx);
    const float sc = Num<float>::exp2i(st.E - En);
    const float2 sc2 = make_float2(sc, sc);
#pragma unroll
    for (int p = 0; p < H; ++p) {
      st.M[p] = fmul2(st.M[p], sc2);
      st.I[p] = fmul2(st.I[p], sc2);
      st.D[p] = fmul2(st.D[p], sc2);
    }
    st.Md *= sc;
    st.Sd *= sc;
    st.acc *= sc;
    st.E = En;
  }
  const float xb = fmaxf(st.M[H - 1].y, fmaxf(st.I[H - 1].y, st.D[H - 1].y));
  const int Eup = __shfl_up_sync(FULL, st.E, 1, L);
  const float xbu = __shfl_up_sync(FULL, xb, 1, L);
  if (zero && t > 0) st.E = Eup - kBias * (K - 1) + (xbu > 0.f ? Num<float>::ilog2(xbu) : 0);
  st.f = Num<float>::exp2i(t == 0 ? -st.E : Eup - st.E - kBias * (K - 1));
}

// Minimum resident blocks per SM the compiler must allow (register budget): rows per lane set
// how many per-row registers a lane holds.
template <typename T, int K>
constexpr int wf_min_blocks() {
  return sizeof(T) == 8 ? 1 : (K <= 8 ? 4 : (K <= 16 ? 3 : 2));
}

// GQ: the batch has a per-base gap-continuation track (row r takes eps_r and beta_r).
template <typename T, int L, int K, bool EXT, bool GQ = false>
__global__ void __launch_bounds__(128, wf_min_blocks<T, K>()) wf_forward(const FwdArgs a) {
  using G_ = TableGeom<T, K>;
  constexpr int G = 32 / L;
  constexpr int VW = G_::VW, LS = G_::LS, CS = G_::CS;
  constexpr unsigned FULL = 0xffffffffu;
  // packed FP32 pairs of rows for the extended-range FP32 tier
  constexpr bool X2 = EXT && sizeof(T) == 4;
  constexpr int H = K / 2;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int t = lane % L, sub = lane / L;
  T *tbl = reinterpret_cast<T *>(smem_raw) + (size_t)warp * kCodes * CS + lane * LS;
  const T eps = sizeof(T) == 4 ? (T)a.eps32 : (T)a.eps64;
  const T beta = sizeof(T) == 4 ? (T)a.beta32 : (T)a.beta64;

  const int64_t count = a.count_dev ? (int64_t)*a.count_dev : a.count;
  const int64_t base = a.offset_dev ? (int64_t)*a.offset_dev : a.list_offset;
  const int64_t nitems = (count + G - 1) / G;
  const int wpb = blockDim.x >> 5;
  int64_t item = (int64_t)blockIdx.x * wpb + warp;
  bool first = true;

  for (;;) {
    if (a.persistent) {
      int it = 0;
      if (lane == 0) it = atomicAdd(a.counter, 1);
      item = __shfl_sync(FULL, it, 0);
    } else if (!first) {
      break;
    }
    first = false;
    if (item >= nitems) break;

    // ---- this lane's pair --------------------------------------------------------------
    const int64_t idx = item * G + sub;
    const bool valid = idx < count;
    int32_t p = -1;
    bool bad = false;
    int m = 0;
    int64_t n = 0, r0 = 0, hs = 0;
    if (valid) {
      p = a.list ? a.list[base + idx] : (int32_t)(base + idx);
      const int32_t ri = a.pair_read[p], hi = a.pair_hap[p];
      if (ri >= 0 && ri < a.n_reads && hi >= 0 && hi < a.n_haps) {
        r0 = a.read_off[ri];
        m = (int)(a.read_off[ri + 1] - r0);
        hs = hap_start(a.hap_off[hi], hi);
        n = a.hap_off[hi + 1] - a.hap_off[hi];
        // reads longer than the group only in row tiles (32 x 16 group, buffer present)
        const bool tiles_ok = L == 32 && K == 16 && a.tilebuf != nullptr && n <= a.tile_cols;
        if (m <= 0 || n <= 0 || (m > L * K && !(tiles_ok && m <= PHMM_MAX_READ_LEN_FWD)))
          bad = true;
      } else {
        bad = true;
      }
#ifdef PHMM_DEBUG
      // the pair's read positions and haplotype codes (with their guards) inside the buffers
      if (!bad && a.dbg_err &&
          (r0 + m > a.dbg_sum_m || hs < kHapGuard ||
           hs + ((n + 15) & ~(int64_t)15) + kHapGuard > a.dbg_hcode_bytes)) {
        atomicOr(a.dbg_err, kDbgPairIndex);
        bad = true;
      }
#endif
      if (bad) {
        m = 0;
        n = 0;
      }
    }
    // Row tiles (Sec. III-C handles reads up to 1,024 bases): the 32 x 16 group scores reads
    // longer than its 512 rows in tiles of 512 rows, top to bottom.  Each tile sweeps every
    // column; its last row (M, I and the third value the lane below takes, with the last
    // lane's exponent) goes column by column to a per-warp buffer, and the next tile's lane 0
    // reads it as the row above its strip.  The top padding sits in the first tile.
    constexpr bool TILED = (L == 32 && K == 16);
    constexpr int LK = L * K;
    const int ntile = TILED ? ((m + LK - 1) / LK > 1 ? (m + LK - 1) / LK : 1) : 1;
    const int npad = ntile * LK - m;
    // K0 * D(0, j), carried in I; the per-lane-exponent tier starts from K0 = 1
    const T bnd = n > 0 ? (EXT ? (T)1 : Num<T>::K0) / (T)n : (T)0;
    constexpr int kBias = EXT ? 2 : 0;
    TileCol<T> *tb_in = nullptr, *tb_out = nullptr;
    if constexpr (TILED) {
      TileCol<T> *tb = reinterpret_cast<TileCol<T> *>(a.tilebuf) +
                       ((size_t)blockIdx.x * wpb + warp) * 2 * (size_t)a.tile_cols;
      tb_in = tb;
      tb_out = tb + a.tile_cols;
    }
    T Sfin = 0;
    int Efin = 0;
    for (int tile = 0; tile < ntile; ++tile) {
    const bool last_tile = tile == ntile - 1;

    // ---- per-row constants and the emission table ---------------------------------------
    // Per-lane-exponent tier: row r of every lane is stored with an extra factor 2^(kBias*r)
    // (folded exactly into the row's emission, delta and I coefficients), which offsets the
    // typical decay of the forward values down the rows so one exponent covers the lane.
    T ap[K], dl[K], zt[K], ei[K], M[K], I[K], D[K];
    T er[GQ ? K : 1];  // per-row gap continuation (track only)
#pragma unroll
    for (int r0v = 0; r0v < K; r0v += VW) {
      T ev[kCodes][VW];
#pragma unroll
      for (int u = 0; u < VW; ++u) {
        if (r0v + u >= K) {  // table padding past the lane's rows
#pragma unroll
          for (int c = 0; c < kCodes; ++c) ev[c][u] = 0;
          continue;
        }
        const int rr = X2 ? x2_row<K>(r0v + u) : r0v + u;  // the row at this table position
        // 0-based read position; < 0: pad row
        const int pos = tile * LK + t * K + rr - npad;
        const T bias = rr ? (T)(1 << kBias) : (T)1;
        M[rr] = 0;
        D[rr] = 0;
        T epr = eps, ber = beta;
        if constexpr (GQ) {
          if (pos >= 0) row_gap<T>(a, r0 + pos, epr, ber);
          er[rr] = epr;
        }
        if (pos >= 0) {
          T Q;
          row_params<T>(a, r0 + pos, ap[rr], dl[rr], zt[rr], Q, GQ ? (double)ber : 0.0);
          const int code = a.rcode[r0 + pos];
          ei[rr] = pos == 0 ? (T)0 : epr * bias;
          dl[rr] *= bias;
          I[rr] = 0;
          const T em = bias * (ber * ((T)1 - Q)), ex = bias * (ber * (Q / (T)3));
#pragma unroll
          for (int c = 0; c < kNull; ++c)
            ev[c][u] = (c == code || c == kN || code == kN) ? em : ex;
          ev[kNull][u] = 0;
        } else {
          ap[rr] = 0;
          dl[rr] = 0;
          zt[rr] = 0;
          ei[rr] = bias;
          I[rr] = bnd * (T)(1ll << (kBias * rr));
#pragma unroll
          for (int c = 0; c < kCodes; ++c) ev[c][u] = 0;
        }
      }
#pragma unroll
      for (int c = 0; c < kCodes; ++c) store_vec<T, VW>(tbl + c * CS + r0v, ev[c]);
    }

    // ---- wavefront ------------------------------------------------------------------------
    int steps = n > 0 ? (int)n + L - 1 : 0;
    steps = __reduce_max_sync(FULL, steps);
    typename std::conditional<X2, WfState2<K>, WfState<T, K>>::type st;
    st.c = kNull;
    st.Md = 0;
    st.Sd = (t == 0 && tile == 0) ? bnd : (T)0;
    st.acc = 0;
    st.f = t == 0 ? (T)1 : Num<T>::exp2i(-kBias * (K - 1));
    st.E = 0;
    float2 ap2[X2 ? H : 1], dl2[X2 ? H : 1], zt2[X2 ? H : 1], ei2[X2 ? H : 1];
    float2 er2[X2 && GQ ? H : 1];
    if constexpr (X2) {
#pragma unroll
      for (int q = 0; q < H; ++q) {
        if constexpr (GQ) er2[q] = make_float2(er[q], er[q + H]);
        st.M[q] = make_float2(M[q], M[q + H]);
        st.I[q] = make_float2(I[q], I[q + H]);
        st.D[q] = make_float2(D[q], D[q + H]);
        ap2[q] = make_float2(ap[q], ap[q + H]);
        dl2[q] = make_float2(dl[q], dl[q + H]);
        zt2[q] = make_float2(zt[q], zt[q + H]);
        ei2[q] = make_float2(ei[q], ei[q + H]);
      }
    } else {
#pragma unroll
      for (int r = 0; r < K; ++r) {
        st.M[r] = M[r];
        st.I[r] = I[r];
        st.D[r] = D[r];
      }
    }
    if constexpr (TILED && EXT) {
      // lane 0 of a lower tile starts at the exponent that brings column 1 of the row above
      // near 1 (its own state is still zero, so this changes nothing else)
      if (tile > 0 && t == 0 && n > 0) {
        const TileCol<T> c1 = tb_in[0];
        const T mx = fmax(c1.M, fmax(c1.I, c1.X));
        st.E = mx > (T)0 ? (int)c1.E - kBias * (K - 1) + Num<T>::ilog2(mx) : 0;
        st.f = Num<T>::exp2i(-st.E);
      }
    }
    const uint4 null16 = make_uint4(0x05050505u, 0x05050505u, 0x05050505u, 0x05050505u);
    // Ramp: the first steps carry the wavefront into every lane; in the per-lane-exponent
    // tier each lane renormalises after every one of them, so a lane adopts its exponent from
    // the values about to reach it rather than from its empty initial state.
    const int ramp = steps < ((L + 15) & ~15) ? steps : ((L + 15) & ~15);
    // The result is taken at the first renormalisation point after the pair's last column:
    // later steps (other pairs of the warp still running) only rescale it by powers of two,
    // which would change the rounding of log10 and make results depend on the packing.
    const int fin = n > 0 ? (int)n + L - 1 : 0;
    bool done = false;
    uint4 hv = null16;
    TileCol<T> cb = {0, 0, 0, 0};  // row above, columns s0+1 .. s0+16 (lane u: column s0+u+1)
    // one step of the tile at 0-based step s (u: step within the current 16-step chunk)
    auto step = [&](int s, int u, int code) {
      T in3[3];
      if constexpr (TILED) {
        T tM = 0, tI, tT;
        if (tile == 0) {
          tI = EXT ? bnd * st.f : bnd;
          tT = EXT ? bnd * st.f : (T)0;
        } else {
          const T bM = __shfl_sync(FULL, cb.M, u), bI = __shfl_sync(FULL, cb.I, u);
          const T bX = __shfl_sync(FULL, cb.X, u), bE = __shfl_sync(FULL, cb.E, u);
          const T cv = EXT ? Num<T>::exp2i((int)bE - st.E - kBias * (K - 1)) : (T)1;
          tM = bM * cv;
          tI = bI * cv;
          tT = bX * cv;
        }
        if constexpr (X2) {
          wf_step_x2<L, K, true, GQ>(st, code, t, bnd, eps, tbl, ap2, dl2, zt2, ei2, tM, tI, tT,
                                     er2);
        } else {
          wf_step<T, L, K, EXT, EXT, false, true, false, GQ>(st, code, t, bnd, eps, tbl, ap, dl,
                                                             zt, ei, in3, tM, tI, tT, er);
        }
        if (!last_tile && t == L - 1) {
          const int64_t j = (int64_t)s + 1 - (L - 1);  // the last lane's column
          if (j >= 1 && j <= n) {
            TileCol<T> o;
            if constexpr (X2) {
              o.M = st.M[H - 1].y;
              o.I = st.I[H - 1].y;
              o.X = fmaf(zt2[H - 1].y, st.D[H - 1].y, st.I[H - 1].y);
            } else {
              o.M = st.M[K - 1];
              o.I = st.I[K - 1];
              o.X = EXT ? st.I[K - 1] + zt[K - 1] * st.D[K - 1] : st.D[K - 1];
            }
            o.E = (T)st.E;
            tb_out[j - 1] = o;
          }
        }
      } else if constexpr (X2) {
        wf_step_x2<L, K, false, GQ>(st, code, t, bnd, eps, tbl, ap2, dl2, zt2, ei2, 0.f, 0.f, 0.f,
                                    er2);
      } else {
        wf_step<T, L, K, EXT, EXT, false, false, false, GQ>(st, code, t, bnd, eps, tbl, ap, dl, zt,
                                                            ei, in3, 0, 0, 0, er);
      }
    };
    auto load_cols = [&](int s0) {
      if constexpr (TILED) {
        if (tile > 0) {
          const int64_t c = (int64_t)s0 + lane;
          cb = (lane < 16 && c < n) ? tb_in[c] : TileCol<T>{0, 0, 0, 0};
        }
      }
    };
    for (int s = 0; s < ramp; ++s) {
      if ((s & 15) == 0) {
        hv = (t == 0 && s < n) ? *reinterpret_cast<const uint4 *>(a.hcode + hs + s) : null16;
        load_cols(s);
      }
      const int q = (s >> 2) & 3;
      const uint32_t w = q == 0 ? hv.x : (q == 1 ? hv.y : (q == 2 ? hv.z : hv.w));
      step(s, s & 15, (w >> (8 * (s & 3))) & 0xff);
      if (!done && s + 1 >= fin) {
        Sfin = st.acc;
        Efin = st.E;
        done = true;
      }
      if constexpr (X2) wf_rescale_x2<L, K, kBias>(st, t);
      else if constexpr (EXT) wf_rescale<T, L, K, kBias>(st, t);
    }
    for (int s0 = ramp; s0 < steps; s0 += 16) {
      hv = (t == 0 && s0 < n) ? *reinterpret_cast<const uint4 *>(a.hcode + hs + s0) : null16;
      load_cols(s0);
#pragma unroll
      for (int u = 0; u < 16; ++u) {
        const uint32_t w = u < 4 ? hv.x : (u < 8 ? hv.y : (u < 12 ? hv.z : hv.w));
        step(s0 + u, u, (w >> (8 * (u & 3))) & 0xff);
      }
      if (!done && s0 + 16 >= fin) {
        Sfin = st.acc;
        Efin = st.E;
        done = true;
      }
      if constexpr (X2) wf_rescale_x2<L, K, kBias>(st, t);
      else if constexpr (EXT) wf_rescale<T, L, K, kBias>(st, t);
    }
    if (!done) {
      Sfin = st.acc;
      Efin = st.E;
    }
    if constexpr (TILED) {  // this tile's last row becomes the next tile's row above
      TileCol<T> *x = tb_in;
      tb_in = tb_out;
      tb_out = x;
      __syncwarp();
    }
    }  // tiles
    const T acc = Sfin;
    const int E = Efin;

    // ---- result: the last lane holds row m ------------------------------------------------
    if (valid && t == L - 1) {
      if (bad) {
        a.out[p] = __longlong_as_double(0x7ff8000000000000ll);
        a.flags[p] = PHMM_FLAG_INVALID;
      } else {
        constexpr double LOG10_2 = 0.301029995663981195213738894724493027;
        const double S = (double)acc;
        const bool finite = S < 1.7976931348623157e308;
        bool ok;
        double lg;
        if constexpr (EXT) {
          ok = S > 0.0 && finite;
          lg = log10(S) + (double)(E - kBias * (K - 1)) * LOG10_2;
        } else if constexpr (sizeof(T) == 4) {
          ok = acc >= kMinAccepted32 && finite;
          lg = log10(S) - 120.0 * LOG10_2;
        } else {
          ok = S >= kMinAccepted64 && finite;
          lg = log10(S) - 1020.0 * LOG10_2;
        }
        if (ok || !a.rescue) {
          a.out[p] = lg;
          a.flags[p] = (uint8_t)(sizeof(T) == 4 ? PHMM_FLAG_FP32 : PHMM_FLAG_RESCUED64) |
                       (uint8_t)(EXT ? PHMM_FLAG_EXTENDED : 0);
        } else {
          const int b = bin64_of_m(m);
          const int pos = atomicAdd(&a.rescue_count[b], 1);
          a.rescue_list[b][pos] = p;
        }
      }
    }
  }
}

template <typename T, int L, int K>
inline size_t wf_smem(int block) {
  return (size_t)(block / 32) * TableGeom<T, K>::warp_bytes;
}

}  // namespace phmm
