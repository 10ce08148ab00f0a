// Adjoint (reverse sweep) of the Pair-HMM forward pass: d log10 L / d(Phred inputs).
//
// Not in the paper (which scores only): the gradient of log10 L with respect to the per-base
// base, insertion and deletion qualities and the gap-continuation penalty, for fitting error
// models.  With adjoints A^ = (dL/dA) / L, the reverse recurrences of Eq. 1-3 are
//   M^(i,j) = a'_{i+1} u(i+1,j+1) + delta_{i+1} I^(i+1,j) + zeta_i D^(i,j+1)   [+1/L, i = m]
//   I^(i,j) = u(i+1,j+1) + eps I^(i+1,j)                                       [+1/L, i = m]
//   D^(i,j) = u(i+1,j+1) + eps D^(i,j+1),        u(i,j) = beta lambda(i,j) M^(i,j)
// and each parameter's partial is a sum over cells of an adjoint times a forward value:
//   alpha_i: sum_j M^ lambda M(i-1,j-1)      beta: sum M^ lambda (I+D)(i-1,j-1)
//   Q_i: sum_j M^ (alpha M + beta (I+D))(i-1,j-1) dlambda/dQ     delta_i: sum_j I^ M(i-1,j)
//   zeta_i: sum_j D^ M(i,j-1)                eps: sum I^ I(i-1,j) + D^ D(i,j-1)
// followed by the chain rule through alpha = 1-(delta+zeta) (or 1-10^(-(iq+dq)/10)),
// beta = 1-eps and P = 10^(-q/10).
//
// GPU design.  The same lane/row decomposition as the forward wavefront, reversed: lane t
// owns K rows, walks the columns from right to left, and exchanges the top row's u and I^
// with the lane above by __shfl_down_sync.  Forward values are recomputed, not stored:
//   phase A  runs the per-lane-exponent FP32 forward and checkpoints every lane's register
//            state at each renormalisation point (every step of the ramp, then every 16
//            steps) into a per-warp scratch slot;
//   phase B  for each segment, last to first: restores the checkpoint, recomputes the
//            segment while recording each step's inputs (a column per step, L2-resident),
//            then runs the adjoint over the segment in reverse and accumulates the partials.
// Adjoints carry their own per-lane power-of-two exponent and the inverse of the forward's
// per-row bias, so forward x adjoint products are posterior-scale numbers; each segment's
// products are scaled by 2^(E_fwd + E_adj).  Per-pair partials are written in FP32 and
// reduced per read in FP64 (grad_reduce.cu).
#include <cstdint>
#include <cstring>
#include <vector>
#include "phmm_internal.cuh"
#include "wavefront.cuh"

struct phmm_plan;

namespace phmm {

const phmm_batch &plan_batch(const phmm_plan *pl);
const phmm_options &plan_options(const phmm_plan *pl);
size_t plan_bwd_offset(const phmm_plan *pl);
int64_t plan_sum_m(const phmm_plan *pl);
int plan_sms(const phmm_plan *pl);
size_t plan_layout_rp(const phmm_plan *pl);
size_t plan_layout_rcode(const phmm_plan *pl);
size_t plan_layout_hcode(const phmm_plan *pl);
size_t plan_layout_bin(const phmm_plan *pl, int which);
double plan_eps64(const phmm_plan *pl);
int64_t plan_n_max(const phmm_plan *pl);
int64_t plan_pair_rows(const phmm_plan *pl);
const int *plan_bwd_cfg_of_m(const phmm_plan *pl);
const std::vector<int> &plan_bwd_used(const phmm_plan *pl);

int launch_binning(const phmm_batch &b, const CfgTable &tab, int32_t *key, int32_t *counts,
                   int32_t *offsets, int32_t *cursor, int32_t *grp_begin, int32_t *grp_count,
                   int32_t *order, cudaStream_t s, int *launches);
int pair_offsets(const phmm_batch &b, char *scratch, int64_t **poff, cudaStream_t s);
int reduce_gradients(const phmm_batch &b, char *scratch, const float *part_bq,
                     const float *part_iq, const float *part_dq, const double *pair_dgcp,
                     float *dbq, float *diq, float *ddq, double *dgcp, cudaStream_t s,
                     int *launches);
size_t reduce_scratch_bytes_aligned(int64_t P, int64_t R);

struct BwdArgs {
  FwdArgs f;               // pair list, inputs and prepared parameters (as the forward)
  const double *dL;        // d(loss)/d(log10 L_p)
  const int64_t *poff;     // partial-gradient offsets per pair
  float *part_bq, *part_iq, *part_dq;
  double *pair_dgcp;
  float *scratch;          // per-warp slots
  int64_t slot_floats;
  int32_t nchk;            // checkpoint capacity per slot
};

// Record widths (floats, multiples of 4) of a checkpoint and of a recorded step.
__host__ __device__ constexpr int ck_width(int K) { return 3 * K + 4; }
__host__ __device__ constexpr int cb_width(int K) { return (3 * K + 6 + 3) & ~3; }

// Records are stored as [record][float4 group][lane], so one warp-wide 128-bit access
// covers 512 contiguous bytes.
template <int W>
__device__ __forceinline__ void rec_store(float *base, int lane, const float (&v)[W]) {
#pragma unroll
  for (int g = 0; g < W / 4; ++g)
    reinterpret_cast<float4 *>(base)[g * 32 + lane] =
        make_float4(v[4 * g], v[4 * g + 1], v[4 * g + 2], v[4 * g + 3]);
}
template <int W>
__device__ __forceinline__ void rec_load(const float *base, int lane, float (&v)[W]) {
#pragma unroll
  for (int g = 0; g < W / 4; ++g) {
    const float4 x = reinterpret_cast<const float4 *>(base)[g * 32 + lane];
    v[4 * g] = x.x;
    v[4 * g + 1] = x.y;
    v[4 * g + 2] = x.z;
    v[4 * g + 3] = x.w;
  }
}

__device__ __forceinline__ int hap_code_at(const uint8_t *hcode, int64_t hs, int64_t n,
                                           int64_t j /* 1-based column */) {
  return (j >= 1 && j <= n) ? (int)hcode[hs + j - 1] : kNull;
}

template <int L, int K>
__global__ void __launch_bounds__(128) wf_backward(const BwdArgs a) {
  using T = float;
  using G_ = TableGeom<float, K>;
  constexpr int G = 32 / L, VW = 4, LS = G_::LS, CS = G_::CS;
  constexpr int kBias = 2;
  constexpr int CKW = ck_width(K), CBW = cb_width(K);
  constexpr unsigned FULL = 0xffffffffu;
  const FwdArgs &fa = a.f;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int t = lane % L, sub = lane / L;
  float *tblE = reinterpret_cast<float *>(smem_raw) + (size_t)warp * 2 * kCodes * CS + lane * LS;
  float *tblW = tblE + kCodes * CS;
  const int wpb = blockDim.x >> 5;
  float *slot = a.scratch + (size_t)(blockIdx.x * wpb + warp) * a.slot_floats;
  float *ckb = slot;
  float *cbb = slot + (size_t)a.nchk * 32 * CKW;
  const T eps = fa.eps32, beta = fa.beta32;

  const int64_t count = *fa.count_dev;
  const int64_t base = *fa.offset_dev;
  const int64_t nitems = (count + G - 1) / G;

  for (;;) {
    int it = 0;
    if (lane == 0) it = atomicAdd(fa.counter, 1);
    const int64_t item = __shfl_sync(FULL, it, 0);
    if (item >= nitems) break;

    // ---- pair and per-row constants ------------------------------------------------------
    const int64_t idx = item * G + sub;
    const bool valid = idx < count;
    int32_t p = -1;
    bool bad = false;
    int m = 0;
    int64_t n = 0, r0 = 0, hs = 0;
    if (valid) {
      p = fa.list[base + idx];
      const int32_t ri = fa.pair_read[p], hi = fa.pair_hap[p];
      if (ri >= 0 && ri < fa.n_reads && hi >= 0 && hi < fa.n_haps) {
        r0 = fa.read_off[ri];
        m = (int)(fa.read_off[ri + 1] - r0);
        hs = hap_start(fa.hap_off[hi], hi);
        n = fa.hap_off[hi + 1] - fa.hap_off[hi];
        if (m <= 0 || m > L * K || n <= 0) bad = true;
      } else {
        bad = true;
      }
      if (bad) {
        m = 0;
        n = 0;
      }
    }
    const int npad = L * K - m;
    const T bnd = n > 0 ? (T)1 / (T)n : (T)0;
    T ap[K], dl[K], zt[K], ei[K], cE[K];
    WfState<T, K> st;
#pragma unroll
    for (int rv = 0; rv < K; rv += VW) {
      T ev[kCodes][VW], wv[kCodes][VW];
#pragma unroll
      for (int u = 0; u < VW; ++u) {
        const int rr = rv + u;
        const int pos = t * K + rr - npad;
        const T bias = rr ? (T)(1 << kBias) : (T)1;
        st.M[rr] = 0;
        st.D[rr] = 0;
        if (pos >= 0) {
          T Q;
          row_params<T>(fa, r0 + pos, ap[rr], dl[rr], zt[rr], Q);
          const int code = fa.rcode[r0 + pos];
          ei[rr] = pos == 0 ? (T)0 : eps * bias;
          cE[rr] = pos == 0 ? (T)0 : bias;
          dl[rr] *= bias;
          st.I[rr] = 0;
          const T em = bias * (beta * ((T)1 - Q)), ex = bias * (beta * (Q / (T)3));
          const T wm = -bias * beta, wx = bias * (beta / (T)3);
#pragma unroll
          for (int c = 0; c < kNull; ++c) {
            const bool mt = c == code || c == kN || code == kN;
            ev[c][u] = mt ? em : ex;
            wv[c][u] = mt ? wm : wx;
          }
          ev[kNull][u] = 0;
          wv[kNull][u] = 0;
        } else {
          ap[rr] = 0;
          dl[rr] = 0;
          zt[rr] = 0;
          ei[rr] = bias;
          cE[rr] = 0;
          st.I[rr] = bnd * (T)(1ll << (kBias * rr));
#pragma unroll
          for (int c = 0; c < kCodes; ++c) ev[c][u] = wv[c][u] = 0;
        }
      }
#pragma unroll
      for (int c = 0; c < kCodes; ++c) {
        store_vec<T, VW>(tblE + c * CS + rv, ev[c]);
        store_vec<T, VW>(tblW + c * CS + rv, wv[c]);
      }
    }
    // coefficients of the row just below the strip (the lower lane's row 0, unbiased)
    const T apb = __shfl_down_sync(FULL, ap[0], 1, L);
    const T dlb = __shfl_down_sync(FULL, dl[0], 1, L);
    const T eib = __shfl_down_sync(FULL, ei[0], 1, L);

    // ---- phase A: forward with checkpoints -------------------------------------------------
    int steps = n > 0 ? (int)n + L - 1 : 0;
    steps = __reduce_max_sync(FULL, steps);
    const int ramp = steps < ((L + 15) & ~15) ? steps : ((L + 15) & ~15);
    const int nq = ramp + (steps - ramp + 15) / 16;
    st.c = kNull;
    st.Md = 0;
    st.Sd = t == 0 ? bnd : (T)0;
    st.acc = 0;
    st.f = t == 0 ? (T)1 : Num<T>::exp2i(-kBias * (K - 1));
    st.E = 0;
    const int fin = n > 0 ? (int)n + L - 1 : 0;
    T Sfin = 0;
    int Efin = 0;
    bool done = false;
    for (int q = 0; q < nq; ++q) {
      const int b = q < ramp ? q : ramp + 16 * (q - ramp);
      const int len = q < ramp ? 1 : 16;
      {
        float ck[CKW];
#pragma unroll
        for (int r = 0; r < K; ++r) {
          ck[r] = st.M[r];
          ck[K + r] = st.I[r];
          ck[2 * K + r] = st.D[r];
        }
        ck[3 * K] = st.Md;
        ck[3 * K + 1] = st.Sd;
        ck[3 * K + 2] = st.f;
        ck[3 * K + 3] = __int_as_float(st.E);
        rec_store<CKW>(ckb + (size_t)q * 32 * CKW, lane, ck);
      }
      for (int u = 0; u < len; ++u) {
        const int s = b + u;  // 0-based step index
        const int cu = (t == 0 && s < n) ? (int)fa.hcode[hs + s] : kNull;
        T in3[3];
        wf_step<T, L, K, true>(st, cu, t, bnd, eps, tblE, ap, dl, zt, ei, in3);
      }
      if (!done && b + len >= fin) {
        Sfin = st.acc;
        Efin = st.E;
        done = true;
      }
      wf_rescale<T, L, K, kBias>(st, t);
    }
    if (!done) {
      Sfin = st.acc;
      Efin = st.E;
    }
    // L = S * 2^(Efin - kBias (K-1)), held by the last lane of the group
    const T S = __shfl_sync(FULL, Sfin, sub * L + L - 1);
    const int ES = __shfl_sync(FULL, Efin, sub * L + L - 1);
    const bool okS = S > (T)0 && S < (T)3.0e38f;

    // ---- phase B: adjoint, segment by segment from the right ------------------------------
    int EB = -st.E;  // adjoint exponent tied to the forward's at the right edge
    T u[K], Db[K], gA[K], gQ[K], gD[K], gZ[K];
#pragma unroll
    for (int r = 0; r < K; ++r) u[r] = Db[r] = gA[r] = gQ[r] = gD[r] = gZ[r] = 0;
    T gS = 0, gE = 0, Itop = 0, diagU = 0;
    T fB = Num<T>::exp2i(__shfl_down_sync(FULL, EB, 1, L) - EB - kBias * (K - 1));
    T seed = okS ? Num<T>::exp2i(-ES - EB) / S : (T)0;

    for (int q = nq - 1; q >= 0; --q) {
      const int b = q < ramp ? q : ramp + 16 * (q - ramp);
      const int len = q < ramp ? 1 : 16;
      {
        float ck[CKW];
        rec_load<CKW>(ckb + (size_t)q * 32 * CKW, lane, ck);
#pragma unroll
        for (int r = 0; r < K; ++r) {
          st.M[r] = ck[r];
          st.I[r] = ck[K + r];
          st.D[r] = ck[2 * K + r];
        }
        st.Md = ck[3 * K];
        st.Sd = ck[3 * K + 1];
        st.f = ck[3 * K + 2];
        st.E = __float_as_int(ck[3 * K + 3]);
      }
      st.c = hap_code_at(fa.hcode, hs, n, (int64_t)b - t);
      const T g = Num<T>::exp2i(st.E + EB);
      // recompute the segment, recording each step's inputs
      for (int u2 = 0; u2 < len; ++u2) {
        const int s = b + u2;
        const int cu = (t == 0 && s < n) ? (int)fa.hcode[hs + s] : kNull;
        float rec[CBW];
#pragma unroll
        for (int r = 0; r < K; ++r) {
          rec[r] = st.M[r];
          rec[K + r] = st.I[r];
          rec[2 * K + r] = st.D[r];
        }
        rec[3 * K] = st.Md;
        rec[3 * K + 1] = st.Sd;
        T in3[3];
        wf_step<T, L, K, true>(st, cu, t, bnd, eps, tblE, ap, dl, zt, ei, in3);
        rec[3 * K + 2] = in3[0];
        rec[3 * K + 3] = in3[1];
        rec[3 * K + 4] = in3[2];
        rec[3 * K + 5] = __int_as_float(st.c);
#pragma unroll
        for (int k = 3 * K + 6; k < CBW; ++k) rec[k] = 0;
        rec_store<CBW>(cbb + (size_t)u2 * 32 * CBW, lane, rec);
      }
      T cM[K], cI[K];
#pragma unroll
      for (int r = 0; r < K; ++r) {
        cM[r] = st.M[r];
        cI[r] = st.I[r];
      }
      // reverse over the segment
      for (int u2 = len - 1; u2 >= 0; --u2) {
        float rec[CBW];
        rec_load<CBW>(cbb + (size_t)u2 * 32 * CBW, lane, rec);
        const int64_t j = (int64_t)b + u2 + 1 - t;  // this lane's column at this step
        const int c = __float_as_int(rec[3 * K + 5]);
        T e[K], w[K];
        load_rows<T, K>(tblE + c * CS, e);
        load_rows<T, K>(tblW + c * CS, w);
        T rU = __shfl_down_sync(FULL, u[0], 1, L);
        T rI = __shfl_down_sync(FULL, Itop, 1, L);
        if (t == L - 1) {
          rU = 0;
          rI = 0;
        } else {
          rU *= fB;
          rI *= fB;
        }
        const T ubK = diagU;
        diagU = rU;
        const T sd = (t == L - 1 && j >= 1 && j <= n) ? seed : (T)0;
        T ub = ubK, Ibl = rI;
        const T Mds = rec[3 * K], Sds = rec[3 * K + 1], inM = rec[3 * K + 2],
                inI = rec[3 * K + 3];
#pragma unroll
        for (int r = K - 1; r >= 0; --r) {
          const T apB = r == K - 1 ? apb : ap[r + 1];
          const T dlB = r == K - 1 ? dlb : dl[r + 1];
          const T eiB = r == K - 1 ? eib : ei[r + 1];
          const T add = r == K - 1 ? sd : (T)0;
          const T Mb = apB * ub + dlB * Ibl + zt[r] * Db[r] + add;
          const T Ib = ub + eiB * Ibl + add;
          const T Dn = ub + eps * Db[r];
          const T un = e[r] * Mb;
          // partials (posterior scale: times g)
          const T Mg = Mb * g, Ig = Ib * g, Dg = Dn * g, ag = un * g;
          const T Mup = r ? rec[r - 1] : Mds;
          const T Sup = r ? rec[K + r - 1] + rec[2 * K + r - 1] : Sds;
          const T Mu = r ? cM[r - 1] : inM;
          const T Iu = r ? cI[r - 1] : inI;
          gA[r] += ag * Mup;
          gS += ag * Sup;
          gQ[r] += (Mg * w[r]) * (ap[r] * Mup + Sup);
          gD[r] += Ig * Mu;
          gE += (Ig * cE[r]) * Iu;
          gZ[r] += Dg * rec[r];
          gE += Dg * rec[2 * K + r];
          ub = u[r];
          u[r] = un;
          Db[r] = Dn;
          Ibl = Ib;
        }
        Itop = Ibl;
#pragma unroll
        for (int r = 0; r < K; ++r) {
          cM[r] = rec[r];
          cI[r] = rec[K + r];
        }
      }
      // renormalise the adjoint state of this lane
      T mx = fmax(Itop, diagU);
#pragma unroll
      for (int r = 0; r < K; ++r) mx = fmax(mx, fmax(u[r], Db[r]));
      if (mx > (T)0) {
        const int En = EB + Num<T>::ilog2(mx);
        const T sc = Num<T>::exp2i(EB - En);
#pragma unroll
        for (int r = 0; r < K; ++r) {
          u[r] *= sc;
          Db[r] *= sc;
        }
        Itop *= sc;
        diagU *= sc;
        EB = En;
      }
      fB = Num<T>::exp2i(__shfl_down_sync(FULL, EB, 1, L) - EB - kBias * (K - 1));
      seed = okS ? Num<T>::exp2i(-ES - EB) / S : (T)0;
    }

    // ---- phase C: chain rule to the Phred inputs, per-pair partials ------------------------
    T gSs = gS, gEs = gE;
#pragma unroll
    for (int o = 1; o < L; o <<= 1) {
      gSs += __shfl_xor_sync(FULL, gSs, o, L);
      gEs += __shfl_xor_sync(FULL, gEs, o, L);
    }
    if (valid && !bad) {
      const double dy = a.dL[p];
      const int64_t po = a.poff[p];
      const T nanv = __int_as_float(0x7fc00000);
#pragma unroll
      for (int r = 0; r < K; ++r) {
        const int pos = t * K + r - npad;
        if (pos < 0) continue;
        const RowParams v = fa.rp[r0 + pos];
        const T del = v.y, zet = v.z, Q = v.w;
        const T gAl = gA[r] / beta;
        const T gDl = gD[r] * (r ? (T)(1 << kBias) : (T)1);
        T db, di, dd;
        if (fa.alpha_mode) {
          const T iq = (T)qual_at(fa.iq, fa.qual_f32, r0 + pos);
          const T dq = (T)qual_at(fa.dq, fa.qual_f32, r0 + pos);
          const T pa = exp10f(-(iq + dq) * 0.1f);
          di = -(gDl * del - gAl * pa) * 0.1f;
          dd = -(gZ[r] * zet - gAl * pa) * 0.1f;
        } else {
          di = -(gDl - gAl) * del * 0.1f;
          dd = -(gZ[r] - gAl) * zet * 0.1f;
        }
        db = -gQ[r] * Q * 0.1f;
        a.part_bq[po + pos] = okS ? (float)(dy * db) : nanv;
        a.part_iq[po + pos] = okS ? (float)(dy * di) : nanv;
        a.part_dq[po + pos] = okS ? (float)(dy * dd) : nanv;
      }
      if (t == 0)
        a.pair_dgcp[p] =
            okS ? -dy * ((double)gEs - (double)gSs / (double)beta) * (double)eps * 0.1 : (double)nanv;
    }
  }
}

// ------------------------------------------------------------------------ host side ------

using BwdKernel = void (*)(const BwdArgs);

static BwdKernel bwd_kernel(int L, int K) {
#define PHMM_BWD_CASE(LL, KK) \
  if (L == LL && K == KK) return wf_backward<LL, KK>;
  PHMM_BWD_CASE(4, 4) PHMM_BWD_CASE(4, 8) PHMM_BWD_CASE(4, 12)
  PHMM_BWD_CASE(8, 4) PHMM_BWD_CASE(8, 8) PHMM_BWD_CASE(8, 12)
  PHMM_BWD_CASE(16, 4) PHMM_BWD_CASE(16, 8) PHMM_BWD_CASE(16, 12)
  PHMM_BWD_CASE(32, 4) PHMM_BWD_CASE(32, 8) PHMM_BWD_CASE(32, 12) PHMM_BWD_CASE(32, 16)
#undef PHMM_BWD_CASE
  return nullptr;
}

static size_t bwd_smem(int K, int block) {
  const int units = K * 4 / 16, LS = (units % 2 == 1) ? K : K + 4;
  return (size_t)(block / 32) * 2 * kCodes * 32 * LS * 4;
}

// Read length -> backward group (rows per lane <= 12 keeps the adjoint state in registers).
int bwd_default_cfg(int m) {
  struct Gp { int cap, L, K; };
  static const Gp order[] = {{16, 4, 4},   {32, 4, 8},    {48, 4, 12},  {64, 8, 8},
                             {96, 8, 12},  {128, 16, 8},  {192, 16, 12}, {256, 32, 8},
                             {384, 32, 12}, {512, 32, 16}};
  for (const Gp &g : order)
    if (m <= g.cap) {
      const int li = g.L == 4 ? 0 : g.L == 8 ? 1 : g.L == 16 ? 2 : 3;
      return li * 5 + (g.K / 4 - 1);
    }
  return 3 * 5 + 3;
}

static int bwd_blocks_per_sm(int cfg, int block) {
  BwdKernel k = bwd_kernel(cfg_lanes(cfg), cfg_rows(cfg));
  if (!k) return 0;
  cudaFuncSetAttribute((const void *)k, cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024);
  int nb = 0;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k, block, bwd_smem(cfg_rows(cfg), block));
  return nb < 1 ? 1 : nb;
}

static int64_t bwd_nchk(int L, int64_t n_max) {
  const int64_t steps = n_max + L - 1 + 16;
  const int64_t ramp = (L + 15) & ~15;
  return ramp + (steps + 15) / 16 + 2;
}

static int64_t bwd_slot_floats(int L, int K, int64_t n_max) {
  return bwd_nchk(L, n_max) * 32 * ck_width(K) + 16 * 32 * cb_width(K);
}

struct BwdLayout {
  size_t part, pdgcp, red, slots, total;
};

static BwdLayout bwd_layout(const phmm_plan *pl) {
  const phmm_batch &b = plan_batch(pl);
  const int block = 32 * plan_options(pl).warps_per_block;
  BwdLayout Lo;
  size_t o = 0;
  auto take = [&](size_t bytes) {
    size_t at = o;
    o = (o + bytes + 255) & ~(size_t)255;
    return at;
  };
  const int64_t rows = plan_pair_rows(pl) + 1;
  Lo.part = take(3 * 4 * (size_t)rows);
  Lo.pdgcp = take(8 * (size_t)(b.n_pairs + 1));
  Lo.red = take(reduce_scratch_bytes_aligned(b.n_pairs, b.n_reads));
  size_t slots = 0;
  for (int cfg : plan_bwd_used(pl)) {
    const int L = cfg_lanes(cfg), K = cfg_rows(cfg);
    const size_t nslot = (size_t)plan_sms(pl) * bwd_blocks_per_sm(cfg, block) * (block / 32);
    const size_t bytes = nslot * 4 * (size_t)bwd_slot_floats(L, K, plan_n_max(pl));
    if (bytes > slots) slots = bytes;
  }
  Lo.slots = take(slots);
  Lo.total = o;
  return Lo;
}

size_t bwd_workspace_bytes(const phmm_plan *pl) { return bwd_layout(pl).total; }

#define CKB(x)                          \
  do {                                  \
    int rc_ = (int)(x);                 \
    if (rc_) return rc_;                \
  } while (0)

// returns a cudaError_t value (0 on success)
int bwd_enqueue_impl(phmm_plan *pl, char *ws, const double *dL, float *dbq, float *diq,
                     float *ddq, double *dgcp, cudaStream_t s, int *launches) {
  const phmm_batch &b = plan_batch(pl);
  const phmm_options &o = plan_options(pl);
  const BwdLayout Lo = bwd_layout(pl);
  char *bw = ws + plan_bwd_offset(pl);
  float *part = (float *)(bw + Lo.part);
  const int64_t rows = plan_pair_rows(pl) + 1;
  float *part_bq = part, *part_iq = part + rows, *part_dq = part + 2 * rows;
  double *pdg = (double *)(bw + Lo.pdgcp);
  char *red = bw + Lo.red;
  int64_t *poff = nullptr;
  CKB(pair_offsets(b, red, &poff, s));
  *launches += 2;
  if (b.n_pairs > 0) {
    // bin pairs by backward group, reusing the forward's sort buffers
    int32_t *counts = (int32_t *)(ws + plan_layout_bin(pl, 0));
    CKB(cudaMemsetAsync(counts, 0, 4 * (size_t)kNumCfg32 * kNBuckets, s));
    CKB(cudaMemsetAsync(ws + plan_layout_bin(pl, 7), 0, 4 * kNumCfg32, s));
    CfgTable tab;
    const int *cm = plan_bwd_cfg_of_m(pl);
    for (int m = 0; m <= PHMM_MAX_READ_LEN; ++m) tab.cfg[m] = (int8_t)cm[m];
    int32_t *grp_begin = (int32_t *)(ws + plan_layout_bin(pl, 4));
    int32_t *grp_count = (int32_t *)(ws + plan_layout_bin(pl, 5));
    int32_t *order = (int32_t *)(ws + plan_layout_bin(pl, 6));
    CKB(launch_binning(b, tab, (int32_t *)(ws + plan_layout_bin(pl, 1)), counts,
                       (int32_t *)(ws + plan_layout_bin(pl, 2)),
                       (int32_t *)(ws + plan_layout_bin(pl, 3)), grp_begin, grp_count, order, s,
                       launches));
    BwdArgs a;
    std::memset(&a, 0, sizeof(a));
    FwdArgs &f = a.f;
    f.pair_read = b.pair_read;
    f.pair_hap = b.pair_hap;
    f.read_off = b.read_off;
    f.hap_off = b.hap_off;
    f.rp = (const RowParams *)(ws + plan_layout_rp(pl));
    f.rcode = (const uint8_t *)(ws + plan_layout_rcode(pl));
    f.hcode = (const uint8_t *)(ws + plan_layout_hcode(pl));
    f.bq = b.base_q;
    f.iq = b.ins_q;
    f.dq = b.del_q;
    f.qual_f32 = b.qual_dtype == PHMM_QUAL_F32;
    f.alpha_mode = b.alpha_mode;
    f.n_reads = b.n_reads;
    f.n_haps = b.n_haps;
    f.list = order;
    const double eps64 = plan_eps64(pl);
    f.eps32 = (float)eps64;
    f.beta32 = (float)(1.0 - eps64);
    f.eps64 = eps64;
    f.beta64 = 1.0 - eps64;
    f.persistent = 1;
    a.dL = dL;
    a.poff = poff;
    a.part_bq = part_bq;
    a.part_iq = part_iq;
    a.part_dq = part_dq;
    a.pair_dgcp = pdg;
    a.scratch = (float *)(bw + Lo.slots);
    const int block = 32 * o.warps_per_block;
    for (int cfg : plan_bwd_used(pl)) {
      const int L = cfg_lanes(cfg), K = cfg_rows(cfg);
      BwdArgs c = a;
      c.f.offset_dev = grp_begin + cfg;
      c.f.count_dev = grp_count + cfg;
      c.f.counter = (int32_t *)(ws + plan_layout_bin(pl, 7)) + cfg;
      c.nchk = (int32_t)bwd_nchk(L, plan_n_max(pl));
      c.slot_floats = bwd_slot_floats(L, K, plan_n_max(pl));
      const int grid = plan_sms(pl) * bwd_blocks_per_sm(cfg, block);
      BwdKernel k = bwd_kernel(L, K);
      if (!k) return (int)cudaErrorInvalidValue;
      k<<<grid, block, bwd_smem(K, block), s>>>(c);
      CKB(cudaGetLastError());
      ++*launches;
    }
  }
  CKB(reduce_gradients(b, red, part_bq, part_iq, part_dq, pdg, dbq, diq, ddq, dgcp, s,
                       launches));
  return 0;
}

}  // namespace phmm
