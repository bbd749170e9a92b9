// Pair test and work-queue build (Algorithm 1 skip rule, Algorithm 2 bitmap and
// map_offset, Section 3.5.1 valid multiplications), for all output tiles of
// all instances of a table at once.
//
// Stream order (after one memset that clears the accumulators):
//   prep      FP64 norm maps -> FP32 mantissa/exponent "screen" forms (B transposed
//             so a tile's k-run is contiguous) and per-CTA sums of squared norms;
//             the last CTA of each instance forms ||A||_F, ||B||_F.
//   count     each CTA owns 32 consecutive tiles of one instance, one warp per
//             tile at a time: lanes test k = lane, lane+32, ...; ballot + popc
//             count the survivors; skipped products are summed for the bounds;
//             split modes bin the surviving products by binade; per-CTA totals
//             and a batch-wide histogram of the per-tile counts.
//   finalize  one CTA per instance over its CTAs' totals: their exclusive scan
//             (the first k_idx slot of each CTA's tiles), statistics and the
//             split-flag binade; the last of these CTAs turns the histogram into
//             the bucket starts of the batch-wide longest-first order.
//   fill      same tile partition: first slots from the CTA base plus a warp
//             scan; the same test again, ballot ranks place the surviving k
//             (increasing) at tile_beg[t] + rank; non-empty tiles take their
//             longest-first slot from a per-count cursor.
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
constexpr int kFinThreads = 1024;

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

// The sum of the relative product p / (||A|| ||B||) = (mA mB mI) 2^(eA + eB + eI).
__device__ __forceinline__ void ext_add_rel(ExtSum& s, Screen a, Screen b, float inv_m, int inv_e) {
  if (a.e == kZeroExp || b.e == kZeroExp) return;
  ext_add(s, __fmul_rn(__fmul_rn(a.m, b.m), inv_m), a.e + b.e + inv_e);
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

// floor(log2(fl(fl(na nb) * inv))) clamped to the flag bins, as the oracle defines it.
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


__device__ __forceinline__ int inst_of_prep_cta(const InstRef& r, int cta) {
  return find_inst(r, cta, [](const Inst& x) { return (int64_t)x.prep0; });
}
__device__ __forceinline__ int inst_of_count_cta(const InstRef& r, int cta) {
  return find_inst(r, cta, [](const Inst& x) { return (int64_t)x.count0; });
}

__global__ void __launch_bounds__(kPrepThreads)
    prep_kernel(InstRef R, PlanBuffers Bf) {
  const int ii = inst_of_prep_cta(R, blockIdx.x);
  const Inst& in = R.at(ii);
  const int bd = in.bd;
  const int64_t total = (int64_t)bd * bd;
  const int lc = blockIdx.x - in.prep0;
  const int nctas = (int)((total + kPrepThreads - 1) / kPrepThreads);
  const int64_t idx = (int64_t)lc * kPrepThreads + threadIdx.x;
  double qa = 0.0, qb = 0.0;
  if (idx < total) {
    const double a = in.nA[idx], b = in.nB[idx];
    Bf.tile_inst[in.tile0 + idx] = ii;
    Bf.sA[in.tile0 + idx] = make_screen(a);
    const int64_t k = idx / bd, j = idx % bd;
    Bf.sBT[in.tile0 + j * bd + k] = make_screen(b);
    qa = a * a;
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

__global__ void __launch_bounds__(kWarpsPerCta * 32)
    count_kernel(InstRef R, PlanBuffers Bf) {
  __shared__ double s_bin_sum[kFlagBins];
  __shared__ int s_bin_cnt[kFlagBins];
  __shared__ long long s_S[kWarpsPerCta];
  __shared__ int s_kmax[kWarpsPerCta], s_ne[kWarpsPerCta];
  __shared__ ExtSum s_b1[kWarpsPerCta], s_b2[kWarpsPerCta];
  const int warp = threadIdx.x / 32, lane = threadIdx.x & 31;
  const int ii = inst_of_count_cta(R, blockIdx.x);
  const Inst& in = R.at(ii);
  const int bd = in.bd, split = in.split, band = in.band;
  const TauScreen T = in.T;
  const TauScreen Thi = in.T_hi;
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
  const int64_t tiles = (int64_t)bd * bd;
  const int64_t lt0 = (int64_t)(blockIdx.x - in.count0) * kTilesPerCta;
  long long wS = 0;
  int wkmax = 0, wne = 0;
  ExtSum wb1{0.0f, 0}, wb2{0.0f, 0};
  for (int r = 0; r < kTileRounds; ++r) {
    const int64_t t = lt0 + warp + (int64_t)r * kWarpsPerCta;
    if (t >= tiles) break;
    const int i = (int)(t / bd), j = (int)(t % bd);
    const Screen* ra = Bf.sA + in.tile0 + (int64_t)i * bd;
    const Screen* rb = Bf.sBT + in.tile0 + (int64_t)j * bd;
    ExtSum sk{0.0f, 0};
    int count = 0;
    int run_bin = kFlagBinMin - 1, run_cnt = 0;
    double run_sum = 0.0;
#pragma unroll 4
    for (int k0 = 0; k0 < bd; k0 += 32) {
      const int k = k0 + lane;
      bool s = false;
      if (k < bd) {
        const Screen a = ra[k], b = rb[k];
        s = survives(a, b, nA + (int64_t)i * bd + k, nB + (int64_t)k * bd + j, T);
        if (s && band) s = !survives(a, b, nA + (int64_t)i * bd + k, nB + (int64_t)k * bd + j, Thi);
        if (!s) {
          ext_add_rel(sk, a, b, inv_m, inv_e);
        } else if (split) {
          const double p = __dmul_rn(nA[(int64_t)i * bd + k], nB[(int64_t)k * bd + j]);
          const int bin = rel_bin_screened(a, b, inv_m, inv_e, nA + (int64_t)i * bd + k,
                                           nB + (int64_t)k * bd + j, inv);
          if (bin != run_bin) {
            if (run_cnt) {
              atomicAdd(&s_bin_sum[run_bin - kFlagBinMin], run_sum);
              atomicAdd(&s_bin_cnt[run_bin - kFlagBinMin], run_cnt);
            }
            run_bin = bin;
            run_cnt = 0;
            run_sum = 0.0;
          }
          run_sum += p;
          ++run_cnt;
        }
      }
      count += __popc(__ballot_sync(0xffffffffu, s));
    }
    if (split && run_cnt) {
      atomicAdd(&s_bin_sum[run_bin - kFlagBinMin], run_sum);
      atomicAdd(&s_bin_cnt[run_bin - kFlagBinMin], run_cnt);
    }
    const ExtSum tot = ext_warp_sum(sk);   // no FP64: the FP64 pipe is narrow here
    if (lane == 0) {
      const int64_t g = in.tile0 + t;
      Bf.cnt[g] = count;
      if (count > 0) atomicAdd(&Bf.bdev->hist[count], 1);
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

// Histogram bin of r = fl(fl(na nb) * inv) (FP64, as the oracle defines it):
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
  const int bd = in.bd;
  const double* nA = in.nA;
  const double* nB = in.nB;
  for (int q = threadIdx.x; q < kHistBins; q += blockDim.x) s_hist[q] = 0u;
  __syncthreads();
  const double inv = in.pd->inv_ab;   // written by the prep kernel
  int inv_e;
  const float inv_m = (float)frexp(inv, &inv_e);
  const int64_t tiles = (int64_t)bd * bd;
  const int64_t lt0 = (int64_t)(blockIdx.x - in.count0) * kTilesPerCta;
  for (int r = 0; r < kTileRounds; ++r) {
    const int64_t t = lt0 + warp + (int64_t)r * kWarpsPerCta;
    if (t >= tiles) break;
    const int i = (int)(t / bd), j = (int)(t % bd);
    const Screen* ra = Bf.sA + in.tile0 + (int64_t)i * bd;
    const Screen* rb = Bf.sBT + in.tile0 + (int64_t)j * bd;
    for (int k0 = 0; k0 < bd; k0 += 32) {
      const int k = k0 + lane;
      const bool act = k < bd;
      int bin = kHistBins;   // inactive lanes: a bin of their own
      if (act)
        bin = hist_bin_screened(ra[k], rb[k], inv_m, inv_e, nA + (int64_t)i * bd + k,
                                nB + (int64_t)k * bd + j, inv);
      const unsigned same = __match_any_sync(0xffffffffu, bin);
      if (act && lane == __ffs(same) - 1) atomicAdd(&s_hist[bin], (unsigned)__popc(same));
    }
  }
  __syncthreads();
  for (int q = threadIdx.x; q < kHistBins; q += blockDim.x)
    if (s_hist[q]) atomicAdd(&in.pd->hist[q], s_hist[q]);
}

// Block-wide exclusive scan of one value per thread (Hillis-Steele in smem).
template <typename V>
__device__ V block_exclusive_scan(V x, V* sh, V& total) {
  const int tid = threadIdx.x;
  sh[tid] = x;
  __syncthreads();
  for (int off = 1; off < kFinThreads; off <<= 1) {
    const V y = tid >= off ? sh[tid - off] : V(0);
    __syncthreads();
    sh[tid] += y;
    __syncthreads();
  }
  const V incl = sh[tid];
  total = sh[kFinThreads - 1];
  __syncthreads();
  return incl - x;
}

__global__ void __launch_bounds__(kFinThreads)
    finalize_kernel(InstRef R, PlanBuffers Bf) {
  __shared__ long long s_ll[kFinThreads];
  __shared__ ExtSum s_x[kFinThreads];
  __shared__ int s_i[kFinThreads];
  const int tid = threadIdx.x;
  const Inst& in = R.at(blockIdx.x);
  const int bd = in.bd;
  const int64_t tiles = (int64_t)bd * bd;
  const int nparts = (int)(((int64_t)bd * bd + kTilesPerCta - 1) / kTilesPerCta);
  PlanDevice* pd = in.pd;

  // per-CTA first k_idx slots: each thread scans a contiguous chunk
  const int chunk = (nparts + kFinThreads - 1) / kFinThreads;
  const int p0 = min(nparts, chunk * tid), p1 = min(nparts, p0 + chunk);
  long long locS = 0;
  int locK = 0, locNE = 0;
  ExtSum locB1{0.0f, 0}, locB2{0.0f, 0};
  for (int q = p0; q < p1; ++q) {
    const int cq = in.count0 + q;
    locS += Bf.part_S[cq];
    locNE += Bf.part_ne[cq];
    locK = max(locK, Bf.part_kmax[cq]);
    ext_add(locB1, Bf.part_b1[cq].m, Bf.part_b1[cq].e);
    ext_add(locB2, Bf.part_b2[cq].m, Bf.part_b2[cq].e);
  }
  long long totS;
  long long baseS = block_exclusive_scan<long long>(locS, s_ll, totS) + in.kidx0;
  for (int q = p0; q < p1; ++q) {
    Bf.cta_base[in.count0 + q] = (int)baseS;
    baseS += Bf.part_S[in.count0 + q];
  }
  long long totNE;
  long long baseNE = block_exclusive_scan<long long>((long long)locNE, s_ll, totNE);
  for (int q = p0; q < p1; ++q) {
    Bf.ne_cta_base[in.count0 + q] = (int)baseNE;
    baseNE += Bf.part_ne[in.count0 + q];
  }
  // max and the extended-range sums (FP32 only)
  s_i[tid] = locK;
  s_x[tid] = locB1;
  __syncthreads();
  for (int s = kFinThreads / 2; s > 0; s >>= 1) {
    if (tid < s) {
      s_i[tid] = max(s_i[tid], s_i[tid + s]);
      ext_add(s_x[tid], s_x[tid + s].m, s_x[tid + s].e);
    }
    __syncthreads();
  }
  const int kmax = s_i[0];
  const ExtSum b1x = s_x[0];
  __syncthreads();
  s_x[tid] = locB2;
  __syncthreads();
  for (int s = kFinThreads / 2; s > 0; s >>= 1) {
    if (tid < s) ext_add(s_x[tid], s_x[tid + s].m, s_x[tid + s].e);
    __syncthreads();
  }
  const ExtSum b2x = s_x[0];
  __syncthreads();

  // split flag binade (one warp): m = the largest mm in [kFlagBinMin - 1, 1]
  // with c1 * sum_{bins < mm} p <= budget; bins are prefix-summed in a fixed
  // order (7 consecutive bins per lane, then a warp scan of the lane totals).
  if (tid < 32) {
    const double ab = pd->norm_a * pd->norm_b;
    const double b1 = ext_value(b1x);
    const double bound2 = sqrt(ext_value(b2x)) * ab;
    constexpr int PER = (kFlagBins + 31) / 32;   // 7
    const int lane = tid;
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
      pd->survivors = totS;
      pd->max_tile = kmax;
      pd->nonempty = (int)totNE;
      pd->bound1 = b1 * ab;
      pd->bound2 = bound2;
      pd->valid_ratio = (double)totS / ((double)bd * (double)bd * (double)bd);
      pd->flag_exp = m;
      pd->flagged = flagged;
    }
  }

  // the last finalize CTA: bucket starts of the batch-wide longest-first order
  __shared__ bool s_last;
  __threadfence();
  __syncthreads();
  if (tid == 0) s_last = atomicAdd(&Bf.bdev->ticket, 1u) == gridDim.x - 1u;
  __syncthreads();
  if (s_last) {
    __threadfence();
    const int c = kMaxBd - tid;      // thread tid owns count c (counts 1 .. kMaxBd)
    const long long h = (c >= 1) ? __ldcg(&Bf.bdev->hist[c]) : 0;
    long long tot_ne;
    const long long start = block_exclusive_scan<long long>(h, s_ll, tot_ne);
    if (c >= 1) Bf.bdev->cursor[c] = (int)start;
    if (tid == 0) Bf.bdev->nonempty = (int)tot_ne;
    // non-empty tiles before each instance (the empty-tile ranks of the fill kernel)
    long long carry = 0;
    for (int i0 = 0; i0 < R.count; i0 += kFinThreads) {
      const int i = i0 + tid;
      const long long v = i < R.count ? (long long)__ldcg(&R.at(i).pd->nonempty) : 0;
      long long tot;
      const long long ex = block_exclusive_scan<long long>(v, s_ll, tot);
      if (i < R.count) R.at(i).pd->ne_base = (int)(carry + ex);
      carry += tot;
    }
  }
}

__global__ void __launch_bounds__(kWarpsPerCta * 32)
    fill_kernel(InstRef R, PlanBuffers Bf) {
  __shared__ int s_beg[kTilesPerCta];
  const int warp = threadIdx.x / 32, lane = threadIdx.x & 31;
  const int ii = inst_of_count_cta(R, blockIdx.x);
  const Inst& in = R.at(ii);
  const int bd = in.bd, split = in.split, quant = in.quant, band = in.band;
  const TauScreen T = in.T;
  const TauScreen Thi = in.T_hi;
  const double* nA = in.nA;
  const double* nB = in.nB;
  const int64_t tiles = (int64_t)bd * bd;
  const int64_t lt0 = (int64_t)(blockIdx.x - in.count0) * kTilesPerCta;
  uint32_t* bitsA = Bf.need_bits;
  uint32_t* bitsB = Bf.need_bits + Bf.need_words;
  if (warp == 0) {   // first k_idx slot of each of the CTA's tiles (kTilesPerCta == 32 lanes)
    const int64_t t = lt0 + lane;
    const int c = t < tiles ? Bf.cnt[in.tile0 + t] : 0;
    int incl = c;
    for (int off = 1; off < 32; off <<= 1) {
      const int y = __shfl_up_sync(0xffffffffu, incl, off);
      if (lane >= off) incl += y;
    }
    const int beg = Bf.cta_base[blockIdx.x] + incl - c;
    s_beg[lane] = beg;
    if (t < tiles) Bf.tile_beg[in.tile0 + t] = beg;
    // empty tiles go after all non-empty ones, in increasing global order: the
    // rank of an empty tile is its number minus the non-empty tiles before it
    const unsigned ne_mask = __ballot_sync(0xffffffffu, c > 0);
    if (t < tiles && c == 0) {
      const int64_t g = in.tile0 + t;
      const int64_t ne_before = (int64_t)in.pd->ne_base + Bf.ne_cta_base[blockIdx.x] +
                                __popc(ne_mask & ((1u << lane) - 1u));
      Bf.order[Bf.bdev->nonempty + (g - ne_before)] = (int)g;
    }
  }
  __syncthreads();
  const double inv = in.pd->inv_ab;
  int inv_e;
  const float inv_m = (float)frexp(inv, &inv_e);
  const int m = in.pd->flag_exp;
  for (int r = 0; r < kTileRounds; ++r) {
    const int lt = warp + r * kWarpsPerCta;
    const int64_t t = lt0 + lt;
    if (t >= tiles) break;
    const int64_t g = in.tile0 + t;
    const int c = Bf.cnt[g];
    if (c == 0) continue;
    if (lane == 0) Bf.order[atomicAdd(&Bf.bdev->cursor[c], 1)] = (int)g;
    const int i = (int)(t / bd), j = (int)(t % bd);
    const Screen* ra = Bf.sA + in.tile0 + (int64_t)i * bd;
    const Screen* rb = Bf.sBT + in.tile0 + (int64_t)j * bd;
    int base = s_beg[lt];
    for (int k0 = 0; k0 < bd; k0 += 32) {
      const int k = k0 + lane;
      bool s = false;
      Screen a{}, b{};
      if (k < bd) {
        a = ra[k];
        b = rb[k];
        s = survives(a, b, nA + (int64_t)i * bd + k, nB + (int64_t)k * bd + j, T);
        if (s && band) s = !survives(a, b, nA + (int64_t)i * bd + k, nB + (int64_t)k * bd + j, Thi);
      }
      const unsigned ball = __ballot_sync(0xffffffffu, s);
      if (s) {
        uint16_t v = (uint16_t)k;
        if (split && rel_bin_screened(a, b, inv_m, inv_e, nA + (int64_t)i * bd + k,
                                      nB + (int64_t)k * bd + j, inv) >= m)
          v |= kSplitFlag;
        Bf.k_idx[base + __popc(ball & ((1u << lane) - 1u))] = v;
      }
      base += __popc(ball);
      if (quant && ball) {
        // list the A and B blocks of surviving triples, each once over the plan
        const int64_t ga = in.tile0 + (int64_t)i * bd + k, gb = in.tile0 + (int64_t)k * bd + j;
        bool newA = false, newB = false;
        if (s) {
          const uint32_t bitA = 1u << (ga & 31), bitB = 1u << (gb & 31);
          newA = (atomicOr(&bitsA[ga >> 5], bitA) & bitA) == 0u;
          newB = (atomicOr(&bitsB[gb >> 5], bitB) & bitB) == 0u;
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

}  // namespace

int prep_ctas_of(int bd) { return (int)(((int64_t)bd * bd + kPrepThreads - 1) / kPrepThreads); }
int count_ctas_of(int bd) { return (int)(((int64_t)bd * bd + kTilesPerCta - 1) / kTilesPerCta); }

size_t plan_layout(Inst* insts, int count, PlanBuffers* b, char* base) {
  int64_t tiles = 0, kslots = 0;
  int prep = 0, cnt = 0;
  for (int i = 0; i < count; ++i) {
    const int64_t bd = insts[i].bd;
    insts[i].tile0 = tiles;
    insts[i].kidx0 = kslots;
    insts[i].prep0 = prep;
    insts[i].count0 = cnt;
    tiles += bd * bd;
    kslots += bd * bd * bd;
    prep += prep_ctas_of((int)bd);
    cnt += count_ctas_of((int)bd);
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
  t.kslots = kslots;
  t.prep_ctas = prep;
  t.count_ctas = cnt;
  t.need_words = (tiles + 31) / 32;
  t.pd = reinterpret_cast<PlanDevice*>(take((size_t)count * sizeof(PlanDevice)));
  t.bdev = reinterpret_cast<BatchDevice*>(take(sizeof(BatchDevice)));
  t.need_bits = reinterpret_cast<uint32_t*>(take((size_t)(2 * t.need_words) * sizeof(uint32_t)));
  t.sA = reinterpret_cast<Screen*>(take((size_t)tiles * sizeof(Screen)));
  t.sBT = reinterpret_cast<Screen*>(take((size_t)tiles * sizeof(Screen)));
  t.part_a = reinterpret_cast<double*>(take((size_t)prep * sizeof(double)));
  t.part_b = reinterpret_cast<double*>(take((size_t)prep * sizeof(double)));
  t.part_S = reinterpret_cast<long long*>(take((size_t)cnt * sizeof(long long)));
  t.part_kmax = reinterpret_cast<int*>(take((size_t)cnt * sizeof(int)));
  t.part_ne = reinterpret_cast<int*>(take((size_t)cnt * sizeof(int)));
  t.part_b1 = reinterpret_cast<ExtSum*>(take((size_t)cnt * sizeof(ExtSum)));
  t.part_b2 = reinterpret_cast<ExtSum*>(take((size_t)cnt * sizeof(ExtSum)));
  t.cta_base = reinterpret_cast<int*>(take((size_t)cnt * sizeof(int)));
  t.ne_cta_base = reinterpret_cast<int*>(take((size_t)cnt * sizeof(int)));
  t.cnt = reinterpret_cast<int*>(take((size_t)tiles * sizeof(int)));
  t.tile_beg = reinterpret_cast<int*>(take((size_t)tiles * sizeof(int)));
  t.order = reinterpret_cast<int*>(take((size_t)tiles * sizeof(int)));
  t.k_idx = reinterpret_cast<uint16_t*>(take((size_t)kslots * sizeof(uint16_t)));
  t.tile_inst = reinterpret_cast<int*>(take((size_t)tiles * sizeof(int)));
  t.need_list = reinterpret_cast<uint32_t*>(take((size_t)(2 * tiles) * sizeof(uint32_t)));
  for (int i = 0; i < count; ++i) insts[i].pd = t.pd ? t.pd + i : nullptr;
  if (b) *b = t;
  return (off + 255) / 256 * 256;
}

InstRef make_ref(const Inst* host_insts, const Inst* dev_table, int count) {
  InstRef r{};
  r.count = count;
  r.table = dev_table;
  if (!dev_table) r.one = host_insts[0];
  return r;
}

cudaError_t run_plan(const InstRef& ref, const PlanBuffers& b, cudaStream_t s) {
  // clear the per-instance statistics and the batch-wide order state (laid
  // out back to back, one memset)
  const size_t clear = reinterpret_cast<const char*>(b.need_bits + 2 * b.need_words) -
                       reinterpret_cast<const char*>(b.pd);
  cudaError_t e = cudaMemsetAsync(b.pd, 0, clear, s);
  if (e != cudaSuccess) return e;
  prep_kernel<<<b.prep_ctas, kPrepThreads, 0, s>>>(ref, b);
  count_kernel<<<b.count_ctas, kWarpsPerCta * 32, 0, s>>>(ref, b);
  finalize_kernel<<<ref.count, kFinThreads, 0, s>>>(ref, b);
  fill_kernel<<<b.count_ctas, kWarpsPerCta * 32, 0, s>>>(ref, b);
  return cudaPeekAtLastError();
}

cudaError_t run_histogram(const InstRef& ref, const PlanBuffers& b, cudaStream_t s) {
  const size_t clear = reinterpret_cast<const char*>(b.need_bits + 2 * b.need_words) -
                       reinterpret_cast<const char*>(b.pd);
  cudaError_t e = cudaMemsetAsync(b.pd, 0, clear, s);
  if (e != cudaSuccess) return e;
  prep_kernel<<<b.prep_ctas, kPrepThreads, 0, s>>>(ref, b);
  hist_kernel<<<b.count_ctas, kWarpsPerCta * 32, 0, s>>>(ref, b);
  return cudaPeekAtLastError();
}

}  // namespace spamm
