// sx_step_common.cuh -- device pieces shared by the step kernels of
// direction-conserving transport (sx_step.cu) and of ballistic and combined
// transport (sx_ballistic.cu): the chemistry of one cell, routing-mask words,
// budget accumulators and ordered packet rounds.
#pragma once

#include "sx_internal.cuh"

namespace sx {

// ----------------------------------------------------------------------------
// Chemistry of one cell over one step (Sect. 4.5): explicit subcycles at
// constant flux F = N_in / dt; each subcycle absorbs F h (1 - e^-tau) photons
// (one ionisation each) and transmits F h e^-tau; its length is
// h = min(t_left, f_c / (Gamma + R)) with Gamma + R = ion / y + alpha_B n_e;
// equilibrium (|dy| <= tol y) keeps the last subcycle's rates for the rest of
// the step.  FP64.  One expm1 per subcycle: e^-tau is 1 + expm1(-tau) (its
// absolute error, 1e-16 of N_in, is what matters for the transmitted
// photons).  f_c / (Gamma + R) = f_c y / (ion + R0 x y) is taken (only where
// it limits the subcycle) with a Newton-Raphson reciprocal, to 1e-15, and
// the products and sums fuse into FMAs: GB300 issues an FP64 warp
// instruction in 16 cycles per SM, and the chemistry's FP64 instructions
// are a large share of a step.  Returns the transmitted fraction
// f = (1/dt) sum e^-tau_k h_k.
// kRec: rec_int receives the recombinations per atom over the step,
// sum R0 x_k^2 h_k (the hold after equilibrium at the last subcycle's rate),
// for diffuse recombination radiation.
// ----------------------------------------------------------------------------
// f_c y / den by a Newton-Raphson reciprocal: an FP32 seed refined twice
// in FP64 (each step squares the relative error: 2^-23 -> 2^-46 -> below an
// ulp); the division itself where den is outside the normal FP32 range.
static __device__ __forceinline__ double fast_quot(double num, double den) {
  const float df = (float)den;
  if (!(df > 1e-37f && df < 1e37f)) return num / den;
  double r = (double)(1.0f / df);
  double e = fma(-den, r, 1.0);
  r = fma(r, e, r);
  e = fma(-den, r, 1.0);
  r = fma(r, e, r);
  return num * r;
}

template <bool kRec = false>
static __device__ double chem_cell(double &y_io, double N_in, double dt, double inv_dt, double invA,
                            double tau_max, double R0, double fc, double tol, int max_sub,
                            int &nsub, int &capped, double *rec_int = nullptr) {
  double y = y_io;
  nsub = 0;
  capped = 0;
  if constexpr (kRec) *rec_int = 0.0;
  if (invA == 0.0) return 1.0;  // no atoms: transparent, nothing to ionise
  const double F = N_in * inv_dt;
  const double Fa = F * invA;
  double t_left = dt;
  double trans_int = 0.0;
  double rec_sum = 0.0;
  while (t_left > 0.0) {
    const double em = expm1(-(tau_max * y));
    const double ab = -em;                   // absorbed fraction
    const double tr = 1.0 + em;              // transmitted fraction
    const double ion = Fa * ab;              // photoionisations per atom per s
    const double x = 1.0 - y;
    const double r0x = R0 * x;
    const double rec = r0x * x;              // recombinations per atom per s
    double h = t_left;
    if (y > 0.0) {
      const double den = fma(r0x, y, ion);
      const double fy = fc * y;
      if (den > 0.0 && fy < den * t_left) h = fast_quot(fy, den);
    } else {
      const double rate = fma(Fa, tau_max, r0x);
      if (rate > 0.0 && fc < rate * t_left) h = fast_quot(fc, rate);
    }
    const double y_new = fma(rec - ion, h, y);
    trans_int = fma(tr, h, trans_int);
    if constexpr (kRec) rec_sum = fma(rec, h, rec_sum);
    t_left = (h == t_left) ? 0.0 : t_left - h;
    nsub++;
    const bool eq = fabs(y_new - y) <= tol * y_new;
    y = y_new;
    if (t_left > 0.0 && (eq || nsub >= max_sub)) {
      if (!eq) capped = 1;
      trans_int = fma(tr, t_left, trans_int);
      if constexpr (kRec) rec_sum = fma(rec, t_left, rec_sum);
      t_left = 0.0;
    }
  }
  y_io = y;
  if constexpr (kRec) *rec_int = rec_sum;
  return trans_int * inv_dt;
}

// ----------------------------------------------------------------------------
// The same subcycles for FP32 transport: rates, subcycle lengths and the
// exponentials in FP32 (the photon field is FP32 already), the neutral
// fraction accumulated in FP64, from float copies of y and x = 1 - y that
// follow the FP32 increments.  The transmitted and the absorbed time
// integrals are summed apart, each accurate where it is small, and the
// returned f is taken from the smaller: e^-tau in thick cells, 1 - absorbed
// in thin ones; *absf is the absorbed fraction, f + absf = 1 up to rounding.
// Fa = F / A, photoionisations per atom per second at full absorption.
// ----------------------------------------------------------------------------
// recf: the recombinations per atom over the step (as rec_int of chem_cell).
static __device__ float chem_cell_f(double &y_io, float Fa, float dt, float tau, float R0, float fc,
                             float tol, int max_sub, int &nsub, int &capped, float &absf,
                             float &recf) {
  double y = y_io;
  float yf = (float)y, xf = (float)(1.0 - y);
  nsub = 0;
  capped = 0;
  float t_left = dt, trans = 0.f, absd = 0.f, recd = 0.f;
  while (t_left > 0.f) {
    const float ty = tau * yf;
    const float ab = -expm1f(-ty);  // absorbed fraction
    const float tr = expf(-ty);     // transmitted fraction
    const float ion = Fa * ab;
    const float r0x = R0 * xf;
    const float rec = r0x * xf;
    float h = t_left;
    if (yf > 0.f) {
      const float den = ion + r0x * yf;
      if (den > 0.f && fc * yf < den * t_left) h = __fdividef(fc * yf, den);
    } else {
      const float rate = Fa * tau + r0x;
      if (rate > 0.f && fc < rate * t_left) h = __fdividef(fc, rate);
    }
    const float dy = (rec - ion) * h;
    y += (double)dy;
    yf += dy;
    xf -= dy;
    trans += tr * h;
    absd += ab * h;
    recd += rec * h;
    t_left = (h == t_left) ? 0.f : t_left - h;
    nsub++;
    const bool eq = fabsf(dy) <= tol * yf;
    if (t_left > 0.f && (eq || nsub >= max_sub)) {
      if (!eq) capped = 1;
      trans += tr * t_left;
      absd += ab * t_left;
      recd += rec * t_left;
      t_left = 0.f;
    }
  }
  y_io = y;
  recf = recd;
  const float inv_dt = 1.f / dt;
  const float fa = absd * inv_dt, ft = trans * inv_dt;
  if (fa < ft) {
    absf = fa;
    return 1.f - fa;
  }
  absf = 1.f - ft;
  return ft;
}

// ----------------------------------------------------------------------------
// Mask words of one edge: bin b is bit b % 32 of word b / 32.  Memory holds
// 1, 2 or 4 words per edge; 65..96 bins are handled as 3 words in registers
// and kept at the 16-byte stride of 4 (the fourth word is zero).
// ----------------------------------------------------------------------------
template <int MW>
__device__ __forceinline__ void load_mask(const uint32_t *__restrict__ M, int64_t e, uint32_t m[MW]) {
  if constexpr (MW == 1) {
    m[0] = __ldg(M + e);
  } else if constexpr (MW == 2) {
    const uint2 v = __ldg(reinterpret_cast<const uint2 *>(M) + e);
    m[0] = v.x; m[1] = v.y;
  } else {
    const uint4 v = __ldg(reinterpret_cast<const uint4 *>(M) + e);
    m[0] = v.x; m[1] = v.y; m[2] = v.z;
    if constexpr (MW == 4) m[3] = v.w;
  }
}
template <int MW>
__device__ __forceinline__ void store_mask(uint32_t *__restrict__ M, int64_t e, const uint32_t m[MW]) {
  if constexpr (MW == 1) {
    M[e] = m[0];
  } else if constexpr (MW == 2) {
    reinterpret_cast<uint2 *>(M)[e] = make_uint2(m[0], m[1]);
  } else if constexpr (MW == 3) {
    reinterpret_cast<uint4 *>(M)[e] = make_uint4(m[0], m[1], m[2], 0u);  // 16-byte stride
  } else {
    reinterpret_cast<uint4 *>(M)[e] = make_uint4(m[0], m[1], m[2], m[3]);
  }
}

// Row stride (elements) of the shared photon tile: odd, so that a lane per
// vertex walking its own row touches 32 distinct banks.
__host__ __device__ __forceinline__ int tile_stride(int nbins) { return nbins | 1; }

// Per-lane budget accumulator: FP64 sum, or float-float in FP32 mode (the
// FP64 pipe is narrow, so FP32-mode tiles combine their partial sums in
// float-float and convert once).
template <typename T>
struct Acc;
template <>
struct Acc<double> {
  double v = 0.0;
  __device__ void add(double x) { v = __dadd_rn(v, x); }
};
template <>
struct Acc<float> {
  FF v{0.f, 0.f};
  __device__ void add(float x) { v = ff_add(v, x); }
};

// A budget term of one lane (the type of Acc<T>::v) and its sums.
template <typename T>
struct Bud;
template <>
struct Bud<double> {
  using type = double;
  __device__ static double add(double a, double b) { return __dadd_rn(a, b); }
  __device__ static double warp_sum(double v) { return warp_sum_d(v); }
  __device__ static double to_double(double v) { return v; }
  __device__ static double shfl_xor(double v, int o) { return __shfl_xor_sync(0xffffffffu, v, o); }
};
template <>
struct Bud<float> {
  using type = FF;
  __device__ static FF add(FF a, FF b) { return ff_add(a, b); }
  __device__ static FF warp_sum(FF v) { return ff_warp_sum(v); }
  __device__ static double to_double(FF v) { return ff_to_double(v); }
  __device__ static FF shfl_xor(FF v, int o) {
    return FF{__shfl_xor_sync(0xffffffffu, v.hi, o), __shfl_xor_sync(0xffffffffu, v.lo, o)};
  }
};

// ----------------------------------------------------------------------------
// The step of one vertex's cell from its N_in (stored units; an FP64 sum, or
// float-float in FP32 mode), Sect. 4.5.  A ghost is another shard's vertex,
// stepped and counted there: nothing here.  A sink absorbs N_in.  Any other
// cell runs the subcycles (FP64; FP32 rates with chem_fp32) from its
// neutral fraction y0, writes y, and with diffuse radiation its
// ground-level recombination photons of the step (dif[v], only where they
// changed from d_prev, the last step's).  Returns the transmitted fraction
// f (0 for ghosts and sinks) and the budget terms: absorbed N_in (1 - f),
// passed to a sink, transmitted N_in f.
// ----------------------------------------------------------------------------
template <typename T>
__device__ __forceinline__ T vertex_chem(const StepArgs &a, const VConst &c, int64_t v, double y0,
                                         typename Bud<T>::type nin_acc, double d_prev, int &nsub,
                                         int &capped, typename Bud<T>::type &babs,
                                         typename Bud<T>::type &bsink, typename Bud<T>::type &btr) {
  T f = T(0);
  if constexpr (sizeof(T) == 8) {
    const double nin = nin_acc;
    if (c.flags & kFlagGhost) {
      // another shard's vertex: stepped and counted there
    } else if (c.flags & kFlagSink) {
      bsink = nin;  // a sink passes nothing on
    } else {
      double yv = y0;
      double d_new = 0.0;  // diffuse radiation: photons made in this step
      if (nin == 0.0 && yv == 1.0) {
        f = 1.0;  // no photons and nothing to recombine: the state is a fixed point
      } else if (a.diffuse) {
        double rec = 0.0;
        f = chem_cell<true>(yv, __dmul_rn(nin, a.punit), a.dt, a.inv_dt, c.invA, c.tau_max, c.R0,
                            a.fc, a.tol, a.max_sub, nsub, capped, &rec);
        a.y[v] = yv;
        if (c.invA != 0.0) d_new = __dmul_rn(a.ground, __ddiv_rn(rec, c.invA)) / a.punit;
      } else {
        f = chem_cell(yv, __dmul_rn(nin, a.punit), a.dt, a.inv_dt, c.invA, c.tau_max, c.R0,
                      a.fc, a.tol, a.max_sub, nsub, capped);
        a.y[v] = yv;
      }
      if (a.diffuse && d_new != d_prev) a.dif[v] = d_new;
      babs = __dmul_rn(nin, __dsub_rn(1.0, f));
      btr = __dmul_rn(nin, f);
    }
  } else {
    const FF nin = nin_acc;
    if (c.flags & kFlagGhost) {
      // another shard's vertex: stepped and counted there
    } else if (c.flags & kFlagSink) {
      bsink = nin;  // a sink passes nothing on
    } else {
      double yv = y0;
      float absf = 0.f;
      double rec = 0.0;  // diffuse radiation: recombinations per atom in this step
      if (nin.hi == 0.f && yv == 1.0) {
        f = 1.f;  // no photons and nothing to recombine: the state is a fixed point
      } else {
        const double Fa = __dmul_rn(__dmul_rn(ff_to_double(nin), a.punit),
                                    __dmul_rn(c.invA, a.inv_dt));
        if (c.invA == 0.0) {
          f = 1.f;  // no atoms: transparent, nothing to ionise
        } else if (a.chem_fp32 && Fa < 1e30 && c.tau_max < 1e30 && c.R0 < 1e30 && a.dt < 1e30) {
          float recf = 0.f;
          f = chem_cell_f(yv, (float)Fa, (float)a.dt, (float)c.tau_max, (float)c.R0,
                          (float)a.fc, (float)a.tol, a.max_sub, nsub, capped, absf, recf);
          rec = recf;
        } else {  // the FP64 subcycles (by default, and where rates leave the FP32 range)
          double fd;
          if (a.diffuse)
            fd = chem_cell<true>(yv, __dmul_rn(ff_to_double(nin), a.punit), a.dt, a.inv_dt,
                                 c.invA, c.tau_max, c.R0, a.fc, a.tol, a.max_sub, nsub,
                                 capped, &rec);
          else
            fd = chem_cell(yv, __dmul_rn(ff_to_double(nin), a.punit), a.dt, a.inv_dt,
                           c.invA, c.tau_max, c.R0, a.fc, a.tol, a.max_sub, nsub, capped);
          f = (float)fd;
          absf = (float)(1.0 - fd);
        }
        a.y[v] = yv;
      }
      if (a.diffuse) {
        const double d_new = c.invA != 0.0 ? __dmul_rn(a.ground, rec / c.invA) / a.punit : 0.0;
        if (d_new != d_prev) a.dif[v] = d_new;
      }
      babs = ff_mul(nin, absf);
      btr = ff_mul(nin, f);
    }
  }
  return f;
}

#ifndef SX_STEP_MIN_BLOCKS
#define SX_STEP_MIN_BLOCKS 6  // resident CTAs per SM the register allocation aims for
#endif

// A step kernel variant works on 32-vertex tiles with G consecutive vertices
// per warp, so kTile / G warps per CTA: G = 4 (8 warps, 6 CTAs/SM) or G = 2
// (16 warps, 3 CTAs/SM), both at 40 registers.
template <int G>
struct Shape {
  static constexpr int kWarps = kTile / G;
  static constexpr int kThreads = 32 * kWarps;
  static constexpr int kMinBlocks = SX_STEP_MIN_BLOCKS * 8 / kWarps;
  static constexpr int kCap = 18 * G;  // out-edges of a group staged at once in phase 3
  static constexpr int kLanesPerVertex = 32 / G;
};

// Adds x to the photons of one bin.  FP64: a plain addition.  FP32: a
// compensated (Kahan-Babuska) addition -- the rounding error of s + x,
// exact by Knuth's two-sum, is accumulated in the bin's compensation word
// *c, which the caller folds into the bin once every packet has arrived.
template <typename T>
__device__ __forceinline__ void bin_add(T *s, T *c, T x) {
  if constexpr (sizeof(T) == 8) {
    *s += x;
  } else {
    const float a = *s;
    const float t = __fadd_rn(a, x);
    const float xb = __fsub_rn(t, a);
    const float err = __fadd_rn(__fsub_rn(a, __fsub_rn(t, xb)), __fsub_rn(x, xb));
    *s = t;
    *c = __fadd_rn(*c, err);
  }
}

// A sum in registers: FP64 plainly, FP32 compensated as bin_add.
template <typename T>
struct CSum {
  T s = T(0);
  __device__ void add(T x) { s += x; }
  __device__ T value() const { return s; }
};
template <>
struct CSum<float> {
  float s = 0.f, c = 0.f;
  __device__ void add(float x) { bin_add(&s, &c, x); }
  __device__ float value() const { return __fadd_rn(s, c); }
};

// One round of photon packets arriving at the vertices of a warp's group:
// lane i adds `val` to bin `key & 127` of group vertex `key >> 7` (if `on`).
// Lanes of equal key add in lane order, one rank at a time, so every bin
// sums its packets in list order.  The rows start at zero; gcomp holds the
// rows' compensation words (FP32, see bin_add), laid out as the rows.
template <typename T, int MW>
__device__ __forceinline__ void add_round(T *grow, T *gcomp, int nbs, uint32_t (*gocc)[MW], bool on,
                                          int key, T val, uint32_t lt_mask) {
  const int k = on ? key : (1 << 12) + (int)(threadIdx.x & 31);  // idle lanes: unique keys
  const uint32_t grp = __match_any_sync(0xffffffffu, k);
  const unsigned rank = __popc(grp & lt_mask);
  const unsigned maxr = __reduce_max_sync(0xffffffffu, on ? rank : 0u);
  const int at = (k >> 7) * nbs + (k & 127);
  for (unsigned r = 0; r <= maxr; ++r) {
    if (on && rank == r) bin_add(grow + at, gcomp + at, val);
    __syncwarp();
  }
  if (on) atomicOr(&gocc[k >> 7][(k & 127) >> 5], 1u << (k & 31));
}

// Bins 0..nbins-1 that fall in mask word w.
__device__ __forceinline__ uint32_t word_bins(int nbins, int w) {
  const int n = nbins - 32 * w;
  return n >= 32 ? 0xffffffffu : (n <= 0 ? 0u : ((1u << n) - 1u));
}

}  // namespace sx
