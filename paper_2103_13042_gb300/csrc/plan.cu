// Pair test and work-queue build (Algorithm 1 skip rule, Algorithm 2 bitmap and
// map_offset, Section 3.5.1 valid multiplications), for all output tiles of
// all instances of a table at once.
//
// Stream order (after one memset that clears the accumulators):
//   prep      FP64 norm maps -> FP32 mantissa/exponent "screen" forms (B transposed
//             so a tile's k-run is contiguous) and per-CTA sums of squared norms;
//             the last CTA of each instance forms ||A||_F, ||B||_F.
//   count     each CTA owns 32 tiles of one instance (consecutive in a grouped
//             raster enumeration: bands of 8 block rows, column by column), one
//             warp per tile at a time: lanes test k = lane, lane+32, ...; the
//             ballot words are kept as the tile's survivor bitmask; skipped
//             products are summed for the bounds; split modes bin the surviving
//             products by binade; per-CTA totals and per-CTA counts of the
//             longest-first buckets (floor(log2 survivors) + 1).
//   finalize  one CTA per instance: one vector scan over its CTAs' totals gives
//             each CTA's first k_idx slot, non-empty rank and bucket slots;
//             statistics and the split-flag binade; the last of these CTAs lays
//             out the batch-wide buckets (largest first) and each instance's
//             place in them.
//   fill      same partition: first slots from the CTA base plus a warp scan;
//             the bitmask words are expanded (ballot ranks place the surviving
//             k, increasing, at tile_beg[t] + rank); each non-empty tile takes
//             its slot in the longest-first order (bucket base + CTA base +
//             rank among the CTA's tiles of the bucket, enumeration order), each
//             empty tile its slot after all non-empty ones.
#include <cstddef>
#include <cstring>
#include <vector>

#include "common.cuh"
#include "plan.cuh"

namespace spamm {

TauScreen make_tau_screen(double tau) {
  TauScreen t{};
  t.tau = tau;
  t.all = tau == 0.0;
  t.none = std::isinf(tau);
  if (!t.all && !t.none) {
    int e;
    double m = std::frexp(tau, &e);
    t.e = e;
    // the FP32 screen is decisive outside [1 - 2^-20, 1 + 2^-20] * m
    t.m_hi = (float)(m * (1.0 + std::ldexp(1.0, -20)));
    t.m_lo = (float)(m * (1.0 - std::ldexp(1.0, -20)));
  }
  return t;
}

namespace {

constexpr int kWarpsPerCta = 8;
constexpr int kTilesPerCta = 32;   // count and fill: 8 warps x 4 tiles
constexpr int kTileRounds = kTilesPerCta / kWarpsPerCta;
constexpr int kPrepThreads = 256;
constexpr int kFinThreads = 512;
constexpr int kGroupRows = 8;      // block rows per band of the tile enumeration
static_assert(kOrderKeys <= kMaxBd + 2 && kOrderKeys <= 32, "order buckets");
static_assert(kTilesPerCta % kGroupRows == 0, "a CTA of a full band covers whole columns");

// Output tile (i, j) at enumeration position `pos` of an instance: bands of
// kGroupRows block rows, column by column inside a band, so that tiles close
// in the enumeration (and so in the multiply's order, which keeps it inside
// a bucket) share block rows of A and block columns of B in L2.
__device__ __forceinline__ void tile_at(int64_t pos64, int bm, int bn, int& i, int& j) {
  const int pos = (int)pos64;              // bm * bn <= 2^22
  const int band_tiles = kGroupRows * bn;
  const int band = pos / band_tiles;
  const int r0 = band * kGroupRows;
  const int rows = min(kGroupRows, bm - r0);
  const int w = pos - band * band_tiles;
  j = w / rows;
  i = r0 + (w - j * rows);
}

// Longest-first bucket of a survivor count c >= 1: floor(log2 c) + 1.  Near-
// equal counts share a bucket, so the order keeps the enumeration's locality.
__device__ __forceinline__ int order_key(int c) { return 32 - __clz(c); }

// Exactly !(na * nb < tau) in FP64, decided in FP32 whenever that is safe.
__device__ __forceinline__ bool survives(Screen a, Screen b, const double* nA_ptr,
                                         const double* nB_ptr, const TauScreen& T) {
  if (T.all) return true;
  if (a.e == kNonFiniteExp || b.e == kNonFiniteExp) return true;  // Inf or NaN product
  if (T.none) return false;
  if (a.e == kZeroExp || b.e == kZeroExp) return false;           // 0 < tau
  const int D = a.e + b.e - T.e;
  if (D >= 3) return true;    // mA mB / mT >= 0.25 * 8 / 1 = 2
  if (D <= -2) return false;  // mA mB / mT <= 1 / 0.5 * 2^-2 = 0.5
  const float scale = D == -1 ? 0.5f : (D == 0 ? 1.0f : (D == 1 ? 2.0f : 4.0f));
  const float q = __fmul_rn(__fmul_rn(a.m, b.m), scale);
  if (q >= T.m_hi) return true;
  if (q < T.m_lo) return false;
  const double p = __dmul_rn(*nA_ptr, *nB_ptr);  // the exact FP64 decision
  return !(p < T.tau);
}

// Extended-range FP32 sums (ExtSum, value m * 2^e): sums of relative products
// far below the FP32 range (decay matrices reach 1e-80 and less) keep ~24
// bits.  Terms below 2^-40 of the running sum are dropped.

// Binade of a positive normal FP32 value.
__device__ __forceinline__ int fexp(float x) {
  return (int)((__float_as_uint(x) >> 23) & 0xffu) - 127;
}

// s += q * 2^E (q > 0 normal).  The magnitudes are compared by their true
// binades; a term below 2^-40 of the other side is dropped.  Mantissas stay
// below 2^41, so the aligned product never leaves the FP32 range.
__device__ __forceinline__ void ext_add(ExtSum& s, float q, int E) {
  if (!(q > 0.0f)) return;
  if (s.m == 0.0f) {
    s.m = q;
    s.e = E;
    return;
  }
  const int ea = s.e + fexp(s.m), eb = E + fexp(q);
  if (eb > ea + 40) {
    s.m = q;
    s.e = E;
    return;
  }
  if (eb < ea - 40) return;
  s.m = __fmaf_rn(q, pow2f(E - s.e), s.m);   // |E - s.e| <= 84
  while (s.m >= 1099511627776.0f) {         // 2^40: renormalise
    s.m *= pow2f(-40);
    s.e += 40;
  }
}

// Per-lane sum of a tile's skipped products q 2^E (q = mA mB in [0.25, 1],
// E = eA + eB), held as S 2^Emax with Emax the largest exponent seen so far;
// terms more than 126 binades below Emax are dropped.  Zero products (m = 0)
// add nothing.  A few FP32/integer operations per term and no branch in the
// common case (E <= Emax).
struct SkipSum {
  float S;
  int Emax;
};
constexpr int kSkipNone = -(1 << 29);

// 2^k for -126 <= k <= 0, and 0 for k < -126.
__device__ __forceinline__ float pow2f_or_zero(int k) {
  return __int_as_float(max(k + 127, 0) << 23);
}

__device__ __forceinline__ void skip_add(SkipSum& s, Screen a, Screen b) {
  const int E = a.e + b.e;
  const float q = __fmul_rn(a.m, b.m);
  const int d = E - s.Emax;
  if (d > 0) {   // a new largest exponent: rescale the running sum
    s.S = __fmul_rn(s.S, pow2f_or_zero(-d));
    s.Emax = E;
  }
  s.S = __fmaf_rn(q, pow2f_or_zero(min(d, 0)), s.S);
}

// The lane's sum as an ExtSum (value m 2^e).
__device__ __forceinline__ ExtSum skip_ext(const SkipSum& s) {
  return s.S > 0.0f ? ExtSum{s.S, s.Emax} : ExtSum{0.0f, 0};
}

// Warp total of ExtSums in one pass: every lane rescales its sum to 2^-40 of
// the warp's largest binade (smaller terms dropped, as ext_add does) and the
// FP32 values are added with xor shuffles (a fixed order).
__device__ __forceinline__ ExtSum ext_warp_sum_fast(ExtSum s) {
  constexpr int kNone = -(1 << 29);
  const int eb = s.m > 0.0f ? s.e + fexp(s.m) : kNone;   // true binade of the lane's sum
  int emax = eb;
  for (int off = 16; off > 0; off >>= 1) emax = max(emax, __shfl_xor_sync(0xffffffffu, emax, off));
  if (emax == kNone) return ExtSum{0.0f, 0};
  float v = 0.0f;
  if (eb >= emax - 40) v = s.m * pow2f(s.e - (emax - 40));   // exponent in [-80, 40]
  for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
  ExtSum r{v, emax - 40};
  while (r.m >= 1099511627776.0f) {   // keep the mantissa below 2^40 (v < 2^89)
    r.m *= pow2f(-40);
    r.e += 40;
  }
  return r;
}

__device__ __forceinline__ ExtSum ext_warp_sum(ExtSum s) {
  for (int off = 16; off > 0; off >>= 1) {
    const float m = __shfl_xor_sync(0xffffffffu, s.m, off);
    const int e = __shfl_xor_sync(0xffffffffu, s.e, off);
    ext_add(s, m, e);
  }
  return s;
}

__device__ __forceinline__ double ext_value(ExtSum s) {
  return s.m == 0.0f ? 0.0 : ldexp((double)s.m, s.e);
}

// floor(log2(fl(fl(na nb) * inv))) clamped to the flag bins: the binade of a relative norm
// product, taken from one FP64 multiply so that every implementation bins it alike.
__device__ __forceinline__ int rel_bin(double p, double inv) {
  const double r = __dmul_rn(p, inv);
  if (!(r > 0.0)) return kFlagBinMin;
  if (isinf(r)) return 1;
  const int b = ilogb(r);
  return b < kFlagBinMin ? kFlagBinMin : (b > 1 ? 1 : b);
}

// The same binade decided from the screen forms in FP32, re-decided in FP64
// only when the FP32 product lies within 2^-20 of a power of two.
__device__ __forceinline__ int rel_bin_screened(Screen a, Screen b, float inv_m, int inv_e,
                                                const double* pa, const double* pb, double inv) {
  if (a.e == kZeroExp || b.e == kZeroExp) return kFlagBinMin;
  if (a.e == kNonFiniteExp || b.e == kNonFiniteExp || !(inv > 0.0))
    return rel_bin(__dmul_rn(*pa, *pb), inv);
  const float q = __fmul_rn(__fmul_rn(a.m, b.m), inv_m);   // in [0.125, 1]
  const uint32_t frac = __float_as_uint(q) & 0x7fffffu;
  if (frac < 8u || frac > 0x7fffffu - 8u) return rel_bin(__dmul_rn(*pa, *pb), inv);
  const int b0 = a.e + b.e + inv_e + ((int)((__float_as_uint(q) >> 23) & 0xffu) - 127);
  return b0 < kFlagBinMin ? kFlagBinMin : (b0 > 1 ? 1 : b0);
}


__host__ __device__ __forceinline__ int64_t prep_units(const Inst& in) {
  const int64_t na = (int64_t)in.bm * in.bk, nb = (int64_t)in.bk * in.bn,
                nt = (int64_t)in.bm * in.bn;
  return na > nb ? (na > nt ? na : nt) : (nb > nt ? nb : nt);
}

}  // namespace

int prep_ctas_of(const Inst& in) {
  return (int)((prep_units(in) + kPrepThreads - 1) / kPrepThreads);
}

namespace {

__device__ __forceinline__ int prep_ctas_dev(const Inst& in) {
  return (int)((prep_units(in) + kPrepThreads - 1) / kPrepThreads);
}

__device__ __forceinline__ int inst_of_prep_cta(const InstRef& r, int cta) {
  return find_inst(r, cta, [](const Inst& x) { return (int64_t)x.prep0; });
}
__device__ __forceinline__ int inst_of_count_cta(const InstRef& r, int cta) {
  return find_inst(r, cta, [](const Inst& x) { return (int64_t)x.count0; });
}

__global__ void __launch_bounds__(kPrepThreads)
    prep_kernel(InstRef R, PlanBuffers Bf) {
  pdl_trigger();
  const int ii = inst_of_prep_cta(R, blockIdx.x);
  const Inst& in = R.at(ii);
  const int64_t na = (int64_t)in.bm * in.bk, nb = (int64_t)in.bk * in.bn,
                nt = (int64_t)in.bm * in.bn;
  const int lc = blockIdx.x - in.prep0;
  const int nctas = prep_ctas_dev(in);
  const int64_t idx = (int64_t)lc * kPrepThreads + threadIdx.x;
  double qa = 0.0, qb = 0.0;
  if (idx < nt) Bf.tile_inst[in.tile0 + idx] = ii;
  if (idx < na) {
    const double a = in.nA[idx];
    Bf.sA[in.ablk0 + idx] = make_screen(a);
    qa = a * a;
  }
  if (idx < nb) {
    const double b = in.nB[idx];
    const int64_t k = idx / in.bn, j = idx % in.bn;
    Bf.sBT[in.bblk0 + j * in.bk + k] = make_screen(b);
    qb = b * b;
  }
  for (int off = 16; off > 0; off >>= 1) {
    qa += __shfl_xor_sync(0xffffffffu, qa, off);
    qb += __shfl_xor_sync(0xffffffffu, qb, off);
  }
  __shared__ double wa[kPrepThreads / 32], wb[kPrepThreads / 32];
  if ((threadIdx.x & 31) == 0) {
    wa[threadIdx.x / 32] = qa;
    wb[threadIdx.x / 32] = qb;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double sa = 0.0, sb = 0.0;
    for (int w = 0; w < kPrepThreads / 32; ++w) {
      sa += wa[w];
      sb += wb[w];
    }
    Bf.part_a[blockIdx.x] = sa;
    Bf.part_b[blockIdx.x] = sb;
  }
  // the last CTA of the instance sums its partials in a fixed order (deterministic)
  __shared__ bool s_last;
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) s_last = atomicAdd(&in.pd->ticket, 1u) == (unsigned)nctas - 1u;
  __syncthreads();
  if (s_last && threadIdx.x < 32) {
    __threadfence();
    const int lane = threadIdx.x;
    double a = 0.0, b = 0.0;
    for (int i = lane; i < nctas; i += 32) {
      a += __ldcg(Bf.part_a + in.prep0 + i);
      b += __ldcg(Bf.part_b + in.prep0 + i);
    }
    for (int off = 16; off > 0; off >>= 1) {
      a += __shfl_xor_sync(0xffffffffu, a, off);
      b += __shfl_xor_sync(0xffffffffu, b, off);
    }
    if (lane == 0) {
      const double na = sqrt(a), nb = sqrt(b), ab = na * nb;
      in.pd->norm_a = na;
      in.pd->norm_b = nb;
      in.pd->inv_ab = ab > 0.0 ? 1.0 / ab : 0.0;
    }
  }
}

// Split modes: adds a surviving product to its binade's shared-memory bin
// (rare: the scale of ||A|| ||B|| is reloaded here rather than kept live).
__device__ __forceinline__ void bin_survivor(Screen a, Screen b, const double* pa, const double* pb,
                                          const PlanDevice* pd, double* bin_sum, int* bin_cnt) {
  const double inv = pd->inv_ab;
  int inv_e;
  const float inv_m = (float)frexp(inv, &inv_e);
  const double p = __dmul_rn(*pa, *pb);
  const int bin = rel_bin_screened(a, b, inv_m, inv_e, pa, pb, inv);
  atomicAdd(&bin_sum[bin - kFlagBinMin], p);
  atomicAdd(&bin_cnt[bin - kFlagBinMin], 1);
}

template <bool SPLIT, bool BAND>
__global__ void __launch_bounds__(kWarpsPerCta * 32, 4)
    count_kernel(InstRef R, PlanBuffers Bf) {
  pdl_wait();
  pdl_trigger();
  __shared__ double s_bin_sum[kFlagBins];
  __shared__ int s_bin_cnt[kFlagBins];
  __shared__ long long s_S[kWarpsPerCta];
  __shared__ int s_kmax[kWarpsPerCta], s_ne[kWarpsPerCta];
  __shared__ ExtSum s_b1[kWarpsPerCta], s_b2[kWarpsPerCta];
  __shared__ int s_keys[kOrderKeys];
  const int warp = threadIdx.x / 32, lane = threadIdx.x & 31;
  if (threadIdx.x < kOrderKeys) s_keys[threadIdx.x] = 0;
  const int ii = inst_of_count_cta(R, blockIdx.x);
  const Inst& in = R.at(ii);
  const int bm = in.bm, bk = in.bk, bn = in.bn;
  const bool split = SPLIT && in.split, band = BAND && in.band;
  const TauScreen T = in.T;
  const double* nA = in.nA;
  const double* nB = in.nB;
  PlanDevice* pd = in.pd;
  if (split) {
    for (int i = threadIdx.x; i < kFlagBins; i += blockDim.x) {
      s_bin_sum[i] = 0.0;
      s_bin_cnt[i] = 0;
    }
  }
  __syncthreads();
  const double inv = pd->inv_ab;   // written by the prep kernel
  int inv_e;
  const float inv_m = (float)frexp(inv, &inv_e);
  const int64_t tiles = (int64_t)bm * bn;
  const int nch = (bk + 31) >> 5;
  const int64_t lt0 = (int64_t)(blockIdx.x - in.count0) * kTilesPerCta;
  // When the CTA's 32 positions lie in one full band they are 8 block rows x
  // 4 block columns (warp w: row r0 + w, columns j0 .. j0 + 3): those 8 rows
  // of A's screens and 4 columns of B's are staged in shared memory with one
  // coalesced load, so each warp meets one memory latency instead of one per
  // tile.  Other CTAs (a ragged last band) read the screens from global memory.
  extern __shared__ Screen s_scr[];   // [8 * bk] A rows, then [4 * bk] B columns
  const int64_t band_tiles = (int64_t)kGroupRows * bn;
  const int64_t band0 = lt0 / band_tiles;
  const int r0 = (int)band0 * kGroupRows;
  const bool staged = band0 == (lt0 + kTilesPerCta - 1) / band_tiles && r0 + kGroupRows <= bm &&
                      lt0 + kTilesPerCta <= tiles;
  const int j0 = (int)((lt0 - band0 * band_tiles) / kGroupRows);
  if (staged) {
    const int na = kGroupRows * bk, nb = kTilesPerCta / kGroupRows * bk;
    const Screen* ga = Bf.sA + in.ablk0 + (int64_t)r0 * bk;
    const Screen* gb = Bf.sBT + in.bblk0 + (int64_t)j0 * bk;
#pragma unroll 4
    for (int x = threadIdx.x; x < na + nb; x += blockDim.x)
      s_scr[x] = x < na ? ga[x] : gb[x - na];
    __syncthreads();
  }
  long long wS = 0;
  int wkmax = 0, wne = 0;
  ExtSum wb1{0.0f, 0}, wb2{0.0f, 0};
  for (int r = 0; r < kTileRounds; ++r) {
    const int64_t pos = lt0 + warp + (int64_t)r * kWarpsPerCta;
    if (pos >= tiles) break;
    int i, j;
    tile_at(pos, bm, bn, i, j);
    const int64_t t = (int64_t)i * bn + j;
    const Screen* ra = staged ? s_scr + (i - r0) * bk : Bf.sA + in.ablk0 + (int64_t)i * bk;
    const Screen* rb = staged ? s_scr + (kGroupRows + j - j0) * bk : Bf.sBT + in.bblk0 + (int64_t)j * bk;
    SkipSum sk{0.0f, kSkipNone};
    int count = 0;
    // the screens of up to kChunks 32-wide chunks of k are loaded together
    // (one latency per group instead of one per chunk)
    constexpr int kChunks = 2;
    for (int kg = 0; kg < bk; kg += 32 * kChunks) {
      Screen av[kChunks], bv[kChunks];
#pragma unroll
      for (int q = 0; q < kChunks; ++q) {
        const int k = kg + 32 * q + lane;
        if (k < bk) {
          av[q] = ra[k];
          bv[q] = rb[k];
        }
      }
#pragma unroll
    for (int q = 0; q < kChunks; ++q) {
      const int k0 = kg + 32 * q;
      if (k0 >= bk) break;   // uniform over the warp
      const int k = k0 + lane;
      bool s = false;
      if (k < bk) {
        const Screen a = av[q], b = bv[q];
        const double* pa = nA + (int64_t)i * bk + k;
        const double* pb = nB + (int64_t)k * bn + j;
        s = survives(a, b, pa, pb, T);
        if (BAND && s && band) s = !survives(a, b, pa, pb, in.T_hi);
        if (!s) {
          skip_add(sk, a, b);
        } else if (split) {
          bin_survivor(a, b, pa, pb, pd, s_bin_sum, s_bin_cnt);
        }
      }
      const unsigned bal = __ballot_sync(0xffffffffu, s);
      count += __popc(bal);
      if (lane == 0) Bf.surv_mask[in.mask0 + t * nch + (k0 >> 5)] = bal;
    }
    }
    // the tile's skipped sum relative to ||A|| ||B|| (times inv = inv_m 2^inv_e);
    // no FP64: the FP64 pipe is narrow here
    ExtSum tot = ext_warp_sum_fast(skip_ext(sk));
    if (tot.m > 0.0f) {
      tot.m = __fmul_rn(tot.m, inv_m);
      tot.e += inv_e;
    }
    if (lane == 0) {
      const int64_t g = in.tile0 + t;
      Bf.cnt[g] = count;
      if (count > 0) atomicAdd(&s_keys[order_key(count)], 1);
      ext_add(wb1, tot.m, tot.e);
      ext_add(wb2, __fmul_rn(tot.m, tot.m), 2 * tot.e);
    }
    wS += count;
    wkmax = max(wkmax, count);
    wne += count > 0;
  }
  if (lane == 0) {
    s_S[warp] = wS;
    s_kmax[warp] = wkmax;
    s_ne[warp] = wne;
    s_b1[warp] = wb1;
    s_b2[warp] = wb2;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    long long S = 0;
    int km = 0, ne = 0;
    ExtSum b1{0.0f, 0}, b2{0.0f, 0};
    for (int w = 0; w < kWarpsPerCta; ++w) {
      S += s_S[w];
      km = max(km, s_kmax[w]);
      ne += s_ne[w];
      ext_add(b1, s_b1[w].m, s_b1[w].e);
      ext_add(b2, s_b2[w].m, s_b2[w].e);
    }
    Bf.part_S[blockIdx.x] = S;
    Bf.part_kmax[blockIdx.x] = km;
    for (int q = 0; q < kOrderKeys; ++q) Bf.part_keys[(int64_t)blockIdx.x * kOrderKeys + q] = s_keys[q];
    Bf.part_ne[blockIdx.x] = ne;
    Bf.part_b1[blockIdx.x] = b1;
    Bf.part_b2[blockIdx.x] = b2;
  }
  if (split) {
    for (int i = threadIdx.x; i < kFlagBins; i += blockDim.x) {
      if (s_bin_cnt[i]) {
        atomicAdd(&pd->bin_sum[i], s_bin_sum[i]);
        atomicAdd(&pd->bin_cnt[i], (unsigned long long)s_bin_cnt[i]);
      }
    }
  }
}

// Histogram bin of r = fl(fl(na nb) * inv) (one FP64 multiply, no other rounding):
// floor(-log2 r) clamped to [0, 63]; r = 0 or NaN goes to bin 63, +Inf to 0.
__device__ __forceinline__ int hist_bin_exact(double p, double inv) {
  const double r = __dmul_rn(p, inv);
  if (!(r > 0.0)) return kHistBins - 1;
  if (isinf(r)) return 0;
  int e;
  const double m = frexp(r, &e);          // r = m 2^e, m in [0.5, 1)
  const int t = -e + (m == 0.5 ? 1 : 0);
  return t < 0 ? 0 : (t > kHistBins - 1 ? kHistBins - 1 : t);
}

// The same bin from the screen forms in FP32; the FP64 form decides whenever
// the FP32 product lies within 2^-20 of a power of two.
__device__ __forceinline__ int hist_bin_screened(Screen a, Screen b, float inv_m, int inv_e,
                                                 const double* pa, const double* pb, double inv) {
  if ((a.e == kZeroExp || b.e == kZeroExp) && inv > 0.0 && !isinf(inv)) return kHistBins - 1;
  if (a.e == kNonFiniteExp || b.e == kNonFiniteExp || a.e == kZeroExp || b.e == kZeroExp ||
      !(inv > 0.0) || isinf(inv))
    return hist_bin_exact(__dmul_rn(*pa, *pb), inv);
  const float q = __fmul_rn(__fmul_rn(a.m, b.m), inv_m);   // in [0.125, 1]
  const uint32_t frac = __float_as_uint(q) & 0x7fffffu;
  if (frac < 8u || frac > 0x7fffffu - 8u) return hist_bin_exact(__dmul_rn(*pa, *pb), inv);
  // r = q' 2^(b0) with q' in (1, 2) not a power of two: floor(-log2 r) = -b0 - 1
  const int b0 = a.e + b.e + inv_e + ((int)((__float_as_uint(q) >> 23) & 0xffu) - 127);
  const int t = -b0 - 1;
  return t < 0 ? 0 : (t > kHistBins - 1 ? kHistBins - 1 : t);
}

// Histogram of every triple of every instance: one warp per output tile,
// lanes over k; equal bins of a warp are merged with match_any before the
// shared-memory atomics, CTA totals go to the instance's global bins.
__global__ void __launch_bounds__(kWarpsPerCta * 32)
    hist_kernel(InstRef R, PlanBuffers Bf) {
  __shared__ unsigned int s_hist[kHistBins];
  const int warp = threadIdx.x / 32, lane = threadIdx.x & 31;
  const int ii = inst_of_count_cta(R, blockIdx.x);
  const Inst& in = R.at(ii);
  const int bk = in.bk, bn = in.bn;
  const double* nA = in.nA;
  const double* nB = in.nB;
  for (int q = threadIdx.x; q < kHistBins; q += blockDim.x) s_hist[q] = 0u;
  __syncthreads();
  const double inv = in.pd->inv_ab;   // written by the prep kernel
  int inv_e;
  const float inv_m = (float)frexp(inv, &inv_e);
  const int64_t tiles = (int64_t)in.bm * bn;
  const int64_t lt0 = (int64_t)(blockIdx.x - in.count0) * kTilesPerCta;
  for (int r = 0; r < kTileRounds; ++r) {
    const int64_t t = lt0 + warp + (int64_t)r * kWarpsPerCta;
    if (t >= tiles) break;
    const int i = (int)(t / bn), j = (int)(t % bn);
    const Screen* ra = Bf.sA + in.ablk0 + (int64_t)i * bk;
    const Screen* rb = Bf.sBT + in.bblk0 + (int64_t)j * bk;
    for (int k0 = 0; k0 < bk; k0 += 32) {
      const int k = k0 + lane;
      const bool act = k < bk;
      int bin = kHistBins;   // inactive lanes: a bin of their own
      if (act)
        bin = hist_bin_screened(ra[k], rb[k], inv_m, inv_e, nA + (int64_t)i * bk + k,
                                nB + (int64_t)k * bn + j, inv);
      const unsigned same = __match_any_sync(0xffffffffu, bin);
      if (act && lane == __ffs(same) - 1) atomicAdd(&s_hist[bin], (unsigned)__popc(same));
    }
  }
  __syncthreads();
  for (int q = threadIdx.x; q < kHistBins; q += blockDim.x)
    if (s_hist[q]) atomicAdd(&in.pd->hist[q], s_hist[q]);
}

// Block-wide exclusive scan of K values per thread at once (one shuffle scan
// per warp, one warp over the warp totals): ex[k] = prefix, total[k] = sum.
// `sh` holds 33 * K ints; every thread of the block calls it.
template <int K>
__device__ void block_scan_vec(const int (&x)[K], int (&ex)[K], int (&total)[K], int* sh) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int nwarps = (int)(blockDim.x >> 5);
  int incl[K];
#pragma unroll
  for (int k = 0; k < K; ++k) incl[k] = x[k];
#pragma unroll
  for (int off = 1; off < 32; off <<= 1) {
#pragma unroll
    for (int k = 0; k < K; ++k) {
      const int y = __shfl_up_sync(0xffffffffu, incl[k], off);
      if (lane >= off) incl[k] += y;
    }
  }
  if (lane == 31)
#pragma unroll
    for (int k = 0; k < K; ++k) sh[warp * K + k] = incl[k];
  __syncthreads();
  if (warp == 0) {
#pragma unroll
    for (int k = 0; k < K; ++k) {
      const int w = lane < nwarps ? sh[lane * K + k] : 0;
      int wi = w;
#pragma unroll
      for (int off = 1; off < 32; off <<= 1) {
        const int y = __shfl_up_sync(0xffffffffu, wi, off);
        if (lane >= off) wi += y;
      }
      sh[lane * K + k] = wi - w;
      if (lane == 31) sh[32 * K + k] = wi;
    }
  }
  __syncthreads();
#pragma unroll
  for (int k = 0; k < K; ++k) {
    ex[k] = sh[warp * K + k] + incl[k] - x[k];
    total[k] = sh[32 * K + k];
  }
  __syncthreads();   // sh is reused by the next scan
}

// One CTA per instance: per-CTA slot bases (survivors, non-empty tiles, order
// buckets) by one vector scan, statistics, skipped bounds and the split-flag
// binade; the last CTA to finish lays out the batch-wide longest-first order.
__global__ void __launch_bounds__(kFinThreads)
    finalize_kernel(InstRef R, PlanBuffers Bf) {
  pdl_wait();
  pdl_trigger();
  constexpr int K = 2 + (kOrderKeys - 1);   // survivors, non-empty, buckets 1 .. kOrderKeys-1
  __shared__ int s_sh[33 * K];
  __shared__ int s_kmax[kFinThreads / 32];
  __shared__ ExtSum s_b1[kFinThreads / 32], s_b2[kFinThreads / 32];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const Inst& in = R.at(blockIdx.x);
  const int nparts = (int)(((int64_t)in.bm * in.bn + kTilesPerCta - 1) / kTilesPerCta);
  PlanDevice* pd = in.pd;

  // each thread takes a contiguous chunk of the instance's count CTAs
  const int chunk = (nparts + kFinThreads - 1) / kFinThreads;
  const int p0 = min(nparts, chunk * tid), p1 = min(nparts, p0 + chunk);
  int loc[K];
#pragma unroll
  for (int k = 0; k < K; ++k) loc[k] = 0;
  int locK = 0;
  ExtSum locB1{0.0f, 0}, locB2{0.0f, 0};
  for (int q = p0; q < p1; ++q) {
    const int cq = in.count0 + q;
    loc[0] += (int)Bf.part_S[cq];   // at most 32 * bk per CTA
    loc[1] += Bf.part_ne[cq];
#pragma unroll
    for (int key = 1; key < kOrderKeys; ++key)
      loc[1 + key] += Bf.part_keys[(int64_t)cq * kOrderKeys + key];
    locK = max(locK, Bf.part_kmax[cq]);
    ext_add(locB1, Bf.part_b1[cq].m, Bf.part_b1[cq].e);
    ext_add(locB2, Bf.part_b2[cq].m, Bf.part_b2[cq].e);
  }
  int ex[K], tot[K];
  block_scan_vec<K>(loc, ex, tot, s_sh);
  {
    int base[K];
#pragma unroll
    for (int k = 0; k < K; ++k) base[k] = ex[k];
    for (int q = p0; q < p1; ++q) {
      const int cq = in.count0 + q;
      Bf.cta_base[cq] = (int)in.kidx0 + base[0];
      base[0] += (int)Bf.part_S[cq];
      Bf.ne_cta_base[cq] = base[1];
      base[1] += Bf.part_ne[cq];
#pragma unroll
      for (int key = 1; key < kOrderKeys; ++key) {
        const int64_t o = (int64_t)cq * kOrderKeys + key;
        Bf.key_cta_base[o] = base[1 + key];
        base[1 + key] += Bf.part_keys[o];
      }
    }
  }
  // max and the extended-range sums (FP32 only): warp shuffles, then warp 0
  for (int off = 16; off > 0; off >>= 1) locK = max(locK, __shfl_xor_sync(0xffffffffu, locK, off));
  locB1 = ext_warp_sum(locB1);
  locB2 = ext_warp_sum(locB2);
  if (lane == 0) {
    s_kmax[warp] = locK;
    s_b1[warp] = locB1;
    s_b2[warp] = locB2;
  }
  __syncthreads();

  // warp 0: totals and the split flag binade m = the largest mm in
  // [kFlagBinMin - 1, 1] with c1 * sum_{bins < mm} p <= budget; bins are
  // prefix-summed in a fixed order (7 consecutive bins per lane, then a warp
  // scan of the lane totals).
  if (warp == 0) {
    int kmax = lane < kFinThreads / 32 ? s_kmax[lane] : 0;
    ExtSum b1x = lane < kFinThreads / 32 ? s_b1[lane] : ExtSum{0.0f, 0};
    ExtSum b2x = lane < kFinThreads / 32 ? s_b2[lane] : ExtSum{0.0f, 0};
    for (int off = 16; off > 0; off >>= 1) kmax = max(kmax, __shfl_xor_sync(0xffffffffu, kmax, off));
    b1x = ext_warp_sum(b1x);
    b2x = ext_warp_sum(b2x);
    const double ab = pd->norm_a * pd->norm_b;
    const double b1 = ext_value(b1x);
    const double bound2 = sqrt(ext_value(b2x)) * ab;
    constexpr int PER = (kFlagBins + 31) / 32;   // 7
    int m = kFlagBinMin - 1;
    long long flagged = 0;
    if (in.split) {
      const double budget = 0.5 * (in.target_rel * ab - bound2);
      double v[PER];
      double run = 0.0;
#pragma unroll
      for (int q = 0; q < PER; ++q) {
        const int b = lane * PER + q;
        v[q] = b < kFlagBins ? pd->bin_sum[b] : 0.0;
        run += v[q];
      }
      double incl = run;
      for (int off = 1; off < 32; off <<= 1) {
        const double y = __shfl_up_sync(0xffffffffu, incl, off);
        if (lane >= off) incl += y;
      }
      double below = incl - run;     // sum of the bins before this lane's first
      int best = kFlagBinMin - 1;
      if (budget >= 0.0) {
#pragma unroll
        for (int q = 0; q < PER; ++q) {
          const int b = lane * PER + q;       // candidate mm = kFlagBinMin + b
          if (b < kFlagBins && in.c1 * below <= budget) best = kFlagBinMin + b;
          below += v[q];
        }
      }
      for (int off = 16; off > 0; off >>= 1) best = max(best, __shfl_xor_sync(0xffffffffu, best, off));
      m = best;
      long long f = 0;
      for (int b = lane; b < kFlagBins; b += 32)
        if (kFlagBinMin + b >= m) f += (long long)pd->bin_cnt[b];
      for (int off = 16; off > 0; off >>= 1) f += __shfl_xor_sync(0xffffffffu, f, off);
      flagged = f;
    }
    if (lane == 0) {
      pd->survivors = tot[0];
      pd->max_tile = kmax;
      pd->nonempty = tot[1];
      for (int key = 1; key < kOrderKeys; ++key) pd->key_tot[key] = tot[1 + key];
      pd->bound1 = b1 * ab;
      pd->bound2 = bound2;
      pd->valid_ratio = (double)tot[0] / ((double)in.bm * (double)in.bk * (double)in.bn);
      pd->flag_exp = m;
      pd->flagged = flagged;
    }
  }

  // one instance: its own totals lay out the order (no other CTA to wait for)
  if (gridDim.x == 1) {
    if (tid == 0) {
      int acc = 0;
      for (int key = kOrderKeys - 1; key >= 1; --key) {   // largest key first
        Bf.bdev->cursor[key] = acc;
        pd->key_base[key] = acc;
        acc += tot[1 + key];
      }
      Bf.bdev->nonempty = acc;
      pd->ne_base = 0;
    }
    return;
  }

  // the last finalize CTA: bucket starts of the batch-wide longest-first
  // order, each instance's first slot in each bucket and its non-empty base
  __shared__ bool s_last;
  __threadfence();
  __syncthreads();
  if (tid == 0) s_last = atomicAdd(&Bf.bdev->ticket, 1u) == gridDim.x - 1u;
  __syncthreads();
  if (s_last) {
    __threadfence();
    constexpr int KB = kOrderKeys;   // buckets 1 .. kOrderKeys-1 and (slot 0) non-empty
    int sum[KB];
#pragma unroll
    for (int k = 0; k < KB; ++k) sum[k] = 0;
    for (int i0 = 0; i0 < R.count; i0 += kFinThreads) {   // pass 1: totals over instances
      const int i = i0 + tid;
      int v[KB], e[KB], t[KB];
#pragma unroll
      for (int k = 0; k < KB; ++k) v[k] = 0;
      if (i < R.count) {
        const PlanDevice* q = R.at(i).pd;
        v[0] = __ldcg(&q->nonempty);
#pragma unroll
        for (int key = 1; key < kOrderKeys; ++key) v[key] = __ldcg(&q->key_tot[key]);
      }
      block_scan_vec<KB>(v, e, t, s_sh);
#pragma unroll
      for (int k = 0; k < KB; ++k) sum[k] += t[k];
    }
    int start[KB];   // start[key]: first slot of the bucket (largest key first)
    {
      int acc = 0;
#pragma unroll
      for (int key = kOrderKeys - 1; key >= 1; --key) {
        start[key] = acc;
        acc += sum[key];
      }
      start[0] = 0;
      if (tid == 0) {
        for (int key = 1; key < kOrderKeys; ++key) Bf.bdev->cursor[key] = start[key];
        Bf.bdev->nonempty = acc;
      }
    }
    int carry[KB];
#pragma unroll
    for (int k = 0; k < KB; ++k) carry[k] = 0;
    for (int i0 = 0; i0 < R.count; i0 += kFinThreads) {   // pass 2: per-instance bases
      const int i = i0 + tid;
      int v[KB], e[KB], t[KB];
#pragma unroll
      for (int k = 0; k < KB; ++k) v[k] = 0;
      if (i < R.count) {
        const PlanDevice* q = R.at(i).pd;
        v[0] = __ldcg(&q->nonempty);
#pragma unroll
        for (int key = 1; key < kOrderKeys; ++key) v[key] = __ldcg(&q->key_tot[key]);
      }
      block_scan_vec<KB>(v, e, t, s_sh);
      if (i < R.count) {
        PlanDevice* q = R.at(i).pd;
        q->ne_base = carry[0] + e[0];
        for (int key = 1; key < kOrderKeys; ++key) q->key_base[key] = start[key] + carry[key] + e[key];
      }
#pragma unroll
      for (int k = 0; k < KB; ++k) carry[k] += t[k];
    }
  }
}

__global__ void __launch_bounds__(kWarpsPerCta * 32, 4)
    fill_kernel(InstRef R, PlanBuffers Bf) {
  pdl_wait();
  pdl_trigger();
  __shared__ int s_beg[kTilesPerCta];
  const int warp = threadIdx.x / 32, lane = threadIdx.x & 31;
  const int ii = inst_of_count_cta(R, blockIdx.x);
  const Inst& in = R.at(ii);
  const int bm = in.bm, bk = in.bk, bn = in.bn, split = in.split, quant = in.quant;
  const double* nA = in.nA;
  const double* nB = in.nB;
  const int64_t tiles = (int64_t)bm * bn;
  const int nch = (bk + 31) >> 5;
  const int64_t lt0 = (int64_t)(blockIdx.x - in.count0) * kTilesPerCta;
  uint32_t* bitsA = Bf.need_bits;
  uint32_t* bitsB = Bf.need_bits + Bf.need_words_a;
  if (warp == 0) {   // first k_idx slot of each of the CTA's tiles (kTilesPerCta == 32 lanes)
    const int64_t pos = lt0 + lane;
    // lane q < kOrderKeys: this CTA's first slot in bucket q (loaded with the counts)
    int key_slot = 0;
    if (lane > 0 && lane < kOrderKeys)
      key_slot = in.pd->key_base[lane] + Bf.key_cta_base[(int64_t)blockIdx.x * kOrderKeys + lane];
    int64_t g = 0;
    int c = 0;
    if (pos < tiles) {
      int i, j;
      tile_at(pos, bm, bn, i, j);
      g = in.tile0 + (int64_t)i * bn + j;
      c = Bf.cnt[g];
    }
    int incl = c;
    for (int off = 1; off < 32; off <<= 1) {
      const int y = __shfl_up_sync(0xffffffffu, incl, off);
      if (lane >= off) incl += y;
    }
    const int beg = Bf.cta_base[blockIdx.x] + incl - c;
    s_beg[lane] = beg;
    if (pos < tiles) Bf.tile_beg[g] = beg;
    // empty tiles go after all non-empty ones, in enumeration order: the rank
    // of an empty tile is its position minus the non-empty tiles before it
    // non-empty tiles: bucket slot = instance base + earlier CTAs + rank among
    // the CTA's lanes of the same bucket (enumeration order inside a bucket)
    const int key = c > 0 ? order_key(c) : 0;
    const unsigned same = __match_any_sync(0xffffffffu, key);
    const int first = __shfl_sync(0xffffffffu, key_slot, key);
    if (c > 0) Bf.order[first + __popc(same & ((1u << lane) - 1u))] = (int)g;
    const unsigned ne_mask = __ballot_sync(0xffffffffu, c > 0);
    if (pos < tiles && c == 0) {
      const int64_t ne_before = (int64_t)in.pd->ne_base + Bf.ne_cta_base[blockIdx.x] +
                                __popc(ne_mask & ((1u << lane) - 1u));
      Bf.order[Bf.bdev->nonempty + (in.tile0 + pos - ne_before)] = (int)g;
    }
  }
  __syncthreads();
  const double inv = in.pd->inv_ab;
  int inv_e;
  const float inv_m = (float)frexp(inv, &inv_e);
  const int m = in.pd->flag_exp;
  // dense skip sets (more than 4 survivors per block on average): most blocks are
  // listed after the first few triples, so a plain read of the bit spares the
  // atomic; on sparse ones the read would only add latency
  const bool read_first =
      quant && in.pd->survivors > 4 * ((int64_t)bm * bk + (int64_t)bk * bn);
  for (int r = 0; r < kTileRounds; ++r) {
    const int lt = warp + r * kWarpsPerCta;
    const int64_t pos = lt0 + lt;
    if (pos >= tiles) break;
    int i, j;
    tile_at(pos, bm, bn, i, j);
    const int64_t g = in.tile0 + (int64_t)i * bn + j;
    const int c = Bf.cnt[g];
    if (c == 0) continue;
    const Screen* ra = Bf.sA + in.ablk0 + (int64_t)i * bk;
    const Screen* rb = Bf.sBT + in.bblk0 + (int64_t)j * bk;
    int base = s_beg[lt];
    // the count kernel's ballots: one word per 32 k, expanded in increasing k
    const uint32_t* mrow = Bf.surv_mask + in.mask0 + ((int64_t)i * bn + j) * nch;
    for (int qg = 0; qg < nch; qg += 4) {
      unsigned words[4];
#pragma unroll
      for (int q = 0; q < 4; ++q) words[q] = qg + q < nch ? __ldg(mrow + qg + q) : 0u;
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const unsigned ball = words[q];
        if (ball == 0u) continue;   // uniform over the warp
        const int k = (qg + q) * 32 + lane;
        const bool s = (ball >> lane) & 1u;
        if (s) {
          uint16_t v = (uint16_t)k;
          if (split && rel_bin_screened(ra[k], rb[k], inv_m, inv_e, nA + (int64_t)i * bk + k,
                                        nB + (int64_t)k * bn + j, inv) >= m)
            v |= kSplitFlag;
          Bf.k_idx[base + __popc(ball & ((1u << lane) - 1u))] = v;
        }
        base += __popc(ball);
        if (quant) {
          // list the A and B blocks of surviving triples, each once over the plan
          const int64_t ga = in.ablk0 + (int64_t)i * bk + k, gb = in.bblk0 + (int64_t)k * bn + j;
          bool newA = false, newB = false;
          if (s) {
            // a bit once set stays set: a plain read from L2 that already shows it
            // spares the atomic (atomics on the same words serialise)
            const uint32_t bitA = 1u << (ga & 31), bitB = 1u << (gb & 31);
            newA = (!read_first || (__ldcg(&bitsA[ga >> 5]) & bitA) == 0u) &&
                   (atomicOr(&bitsA[ga >> 5], bitA) & bitA) == 0u;
            newB = (!read_first || (__ldcg(&bitsB[gb >> 5]) & bitB) == 0u) &&
                   (atomicOr(&bitsB[gb >> 5], bitB) & bitB) == 0u;
          }
          const unsigned ma = __ballot_sync(0xffffffffu, newA), mb = __ballot_sync(0xffffffffu, newB);
          if (ma | mb) {
            int nb = 0;
            if (lane == 0) nb = atomicAdd(&Bf.bdev->need_count, __popc(ma) + __popc(mb));
            nb = __shfl_sync(0xffffffffu, nb, 0);
            const unsigned lt = (1u << lane) - 1u;
            if (newA) Bf.need_list[nb + __popc(ma & lt)] = (uint32_t)ga;
            if (newB) Bf.need_list[nb + __popc(ma) + __popc(mb & lt)] = (uint32_t)gb | 0x80000000u;
          }
        }
      }
    }
  }
}

}  // namespace

int count_ctas_of(const Inst& in) {
  return (int)(((int64_t)in.bm * in.bn + kTilesPerCta - 1) / kTilesPerCta);
}

void set_general(Inst& in, int64_t m, int64_t kd, int64_t n, int64_t lda, int64_t ldb,
                 int64_t ldc, float alpha, float beta, int leaf) {
  in.m = m;
  in.kd = kd;
  in.n = n;
  in.lda = lda;
  in.ldb = ldb;
  in.ldc = ldc;
  in.bm = (int)num_blocks(m, leaf);
  in.bk = (int)num_blocks(kd, leaf);
  in.bn = (int)num_blocks(n, leaf);
  in.alpha = alpha;
  in.beta = beta;
}

void set_square(Inst& in, int64_t n, int leaf) { set_general(in, n, n, n, n, n, n, 1.0f, 0.0f, leaf); }

size_t plan_layout(Inst* insts, int count, PlanBuffers* b, char* base, bool norm_parts) {
  int64_t tiles = 0, ablks = 0, bblks = 0, kslots = 0, mwords = 0, groups = 0;
  int prep = 0, cnt = 0, max_bk = 0;
  for (int i = 0; i < count; ++i) {
    Inst& in = insts[i];
    const int64_t bm = in.bm, bk = in.bk, bn = in.bn;
    max_bk = max_bk > (int)bk ? max_bk : (int)bk;
    in.tile0 = tiles;
    in.ablk0 = ablks;
    in.bblk0 = bblks;
    in.kidx0 = kslots;
    in.mask0 = mwords;
    in.grp0 = groups;
    in.prep0 = prep;
    in.count0 = cnt;
    tiles += bm * bn;
    ablks += bm * bk;
    bblks += bk * bn;
    kslots += bm * bk * bn;
    mwords += bm * bn * ((bk + 31) / 32);
    groups += bm * ((bn + kGroupTiles - 1) / kGroupTiles);
    prep += prep_ctas_of(in);
    cnt += count_ctas_of(in);
  }
  size_t off = 0;
  auto take = [&](size_t bytes) {
    off = (off + 255) / 256 * 256;
    char* p = base ? base + off : nullptr;
    off += bytes;
    return p;
  };
  PlanBuffers t{};
  t.tiles = tiles;
  t.groups = groups;
  t.ablks = ablks;
  t.bblks = bblks;
  t.kslots = kslots;
  t.prep_ctas = prep;
  t.count_ctas = cnt;
  t.max_bk = max_bk;
  t.need_words_a = (ablks + 31) / 32;
  t.need_words_b = (bblks + 31) / 32;
  t.pd = reinterpret_cast<PlanDevice*>(take((size_t)count * sizeof(PlanDevice)));
  t.bdev = reinterpret_cast<BatchDevice*>(take(sizeof(BatchDevice)));
  t.need_bits = reinterpret_cast<uint32_t*>(
      take((size_t)(t.need_words_a + t.need_words_b) * sizeof(uint32_t)));
  t.sA = reinterpret_cast<Screen*>(take((size_t)ablks * sizeof(Screen)));
  t.sBT = reinterpret_cast<Screen*>(take((size_t)bblks * sizeof(Screen)));
  t.part_a = reinterpret_cast<double*>(take((size_t)prep * sizeof(double)));
  t.part_b = reinterpret_cast<double*>(take((size_t)prep * sizeof(double)));
  t.part_S = reinterpret_cast<long long*>(take((size_t)cnt * sizeof(long long)));
  t.part_kmax = reinterpret_cast<int*>(take((size_t)cnt * sizeof(int)));
  t.part_ne = reinterpret_cast<int*>(take((size_t)cnt * sizeof(int)));
  t.part_b1 = reinterpret_cast<ExtSum*>(take((size_t)cnt * sizeof(ExtSum)));
  t.part_b2 = reinterpret_cast<ExtSum*>(take((size_t)cnt * sizeof(ExtSum)));
  t.cta_base = reinterpret_cast<int*>(take((size_t)cnt * sizeof(int)));
  t.ne_cta_base = reinterpret_cast<int*>(take((size_t)cnt * sizeof(int)));
  t.part_keys = reinterpret_cast<int*>(take((size_t)cnt * kOrderKeys * sizeof(int)));
  t.key_cta_base = reinterpret_cast<int*>(take((size_t)cnt * kOrderKeys * sizeof(int)));
  t.cnt = reinterpret_cast<int*>(take((size_t)tiles * sizeof(int)));
  t.tile_beg = reinterpret_cast<int*>(take((size_t)tiles * sizeof(int)));
  t.order = reinterpret_cast<int*>(take((size_t)tiles * sizeof(int)));
  t.k_idx = reinterpret_cast<uint16_t*>(take((size_t)kslots * sizeof(uint16_t)));
  t.tile_inst = reinterpret_cast<int*>(take((size_t)tiles * sizeof(int)));
  t.surv_mask = reinterpret_cast<uint32_t*>(take((size_t)mwords * sizeof(uint32_t)));
  t.need_list = reinterpret_cast<uint32_t*>(take((size_t)(ablks + bblks) * sizeof(uint32_t)));
  t.norm_part = norm_parts ? take((size_t)tiles * kMaxEpiWarps * sizeof(NormPart)) : nullptr;
  for (int i = 0; i < count; ++i) insts[i].pd = t.pd ? t.pd + i : nullptr;
  if (b) *b = t;
  return (off + 255) / 256 * 256;
}

InstRef make_ref(const Inst* host_insts, const Inst* dev_table, int count) {
  InstRef r{};
  r.count = count;
  r.table = dev_table;
  if (!dev_table) r.one = host_insts[0];
  for (int i = 0; i < count; ++i) {
    r.any_split |= host_insts[i].split != 0;
    r.any_band |= host_insts[i].band != 0;
    r.any_norm_out |= host_insts[i].nC != nullptr;
    r.any_scaled |= host_insts[i].alpha != 1.0f || host_insts[i].beta != 0.0f;
  }
  return r;
}

// The count kernel with its staged screens: 12 * max_bk screens of shared memory.
cudaError_t launch_count(const InstRef& ref, const PlanBuffers& b, cudaStream_t s) {
  const size_t smem = (size_t)(kGroupRows + kTilesPerCta / kGroupRows) * b.max_bk * sizeof(Screen);
  auto* kern = ref.any_band ? (ref.any_split ? count_kernel<true, true> : count_kernel<false, true>)
                            : (ref.any_split ? count_kernel<true, false> : count_kernel<false, false>);
  {   // opt in to the largest size once per device and variant (static shared memory counts too)
    static bool opted[64][4] = {};
    const int v = (ref.any_band ? 2 : 0) + (ref.any_split ? 1 : 0);
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev >= 0 && dev < 64 && !opted[dev][v]) {
      e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                               (int)((kGroupRows + kTilesPerCta / kGroupRows) * kMaxBd * sizeof(Screen)));
      if (e != cudaSuccess) return e;
      opted[dev][v] = true;
    }
  }
  return launch_pdl(kern, dim3(b.count_ctas), dim3(kWarpsPerCta * 32), smem, s, ref, b);
}

cudaError_t run_plan_count_half(const InstRef& ref, const PlanBuffers& b, cudaStream_t s) {
  // clear the per-instance statistics, the batch-wide order state and the
  // needed-block bits (laid out back to back, one memset)
  const size_t clear =
      reinterpret_cast<const char*>(b.need_bits + b.need_words_a + b.need_words_b) -
      reinterpret_cast<const char*>(b.pd);
  cudaError_t e = cudaMemsetAsync(b.pd, 0, clear, s);
  if (e != cudaSuccess) return e;
  prep_kernel<<<b.prep_ctas, kPrepThreads, 0, s>>>(ref, b);
  e = launch_count(ref, b, s);
  if (e != cudaSuccess) return e;
  return cudaPeekAtLastError();
}

cudaError_t run_plan_queue_half(const InstRef& ref, const PlanBuffers& b, cudaStream_t s) {
  cudaError_t e = launch_pdl(finalize_kernel, dim3(ref.count), dim3(kFinThreads), 0, s, ref, b);
  if (e == cudaSuccess)
    e = launch_pdl(fill_kernel, dim3(b.count_ctas), dim3(kWarpsPerCta * 32), 0, s, ref, b);
  return e;
}

cudaError_t run_plan(const InstRef& ref, const PlanBuffers& b, cudaStream_t s) {
  cudaError_t e = run_plan_count_half(ref, b, s);
  if (e == cudaSuccess) e = run_plan_queue_half(ref, b, s);
  return e;
}

cudaError_t run_plan_count(const InstRef& ref, const PlanBuffers& b, cudaStream_t s) {
  const size_t clear =
      reinterpret_cast<const char*>(b.need_bits + b.need_words_a + b.need_words_b) -
      reinterpret_cast<const char*>(b.pd);
  cudaError_t e = cudaMemsetAsync(b.pd, 0, clear, s);
  if (e != cudaSuccess) return e;
  prep_kernel<<<b.prep_ctas, kPrepThreads, 0, s>>>(ref, b);
  e = launch_count(ref, b, s);
  if (e != cudaSuccess) return e;
  e = launch_pdl(finalize_kernel, dim3(ref.count), dim3(kFinThreads), 0, s, ref, b);
  if (e != cudaSuccess) return e;
  return cudaPeekAtLastError();
}

cudaError_t run_histogram(const InstRef& ref, const PlanBuffers& b, cudaStream_t s) {
  const size_t clear =
      reinterpret_cast<const char*>(b.need_bits + b.need_words_a + b.need_words_b) -
      reinterpret_cast<const char*>(b.pd);
  cudaError_t e = cudaMemsetAsync(b.pd, 0, clear, s);
  if (e != cudaSuccess) return e;
  prep_kernel<<<b.prep_ctas, kPrepThreads, 0, s>>>(ref, b);
  hist_kernel<<<b.count_ctas, kWarpsPerCta * 32, 0, s>>>(ref, b);
  return cudaPeekAtLastError();
}

}  // namespace spamm
