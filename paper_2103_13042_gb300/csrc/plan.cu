// Pair test and work-queue build (Algorithm 1 skip rule, Algorithm 2 bitmap and
// map_offset, Section 3.5.1 valid multiplications), for all output tiles at once.
//
// Kernels, in stream order:
//   prep      FP64 norm maps -> FP32 mantissa/exponent "screen" forms (B transposed
//             so a tile's k-run is contiguous) and partial sums of squared norms.
//   norms     ||A||_F, ||B||_F and 1/(||A|| ||B||); clears the accumulators.
//   count     one warp per output tile (i, j): lanes test k = lane, lane+32, ...;
//             ballot + popc count the survivors; skipped products are summed
//             for the bounds; split modes bin surviving products by binade.
//   finalize  one CTA: exclusive scan of the counts (CSR tile_ptr), statistics,
//             the split-flag binade, and the longest-first tile order.
//   fill      one warp per non-empty tile: the same test again; ballot ranks
//             place the surviving k (increasing) at tile_ptr[t] + rank.
#include "common.cuh"
#include "plan.cuh"

namespace spamm {
namespace {

constexpr int kWarpsPerCta = 8;

struct TauScreen {
  double tau;
  float m_lo, m_hi;
  int32_t e;
  int all;   // tau == 0: every triple survives
  int none;  // tau == +Inf: only non-finite products survive
};

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

// Extended-range FP32 sum: value = m * 2^e with an integer exponent, so sums of
// relative products far below the FP32 range (decay matrices reach 1e-80 and
// less) keep ~24 bits.  Terms below 2^-40 of the running sum are dropped.
struct ExtSum {
  float m;
  int e;
};

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

__global__ void prep_kernel(const double* __restrict__ nA, const double* __restrict__ nB, int bd,
                            Screen* __restrict__ sA, Screen* __restrict__ sBT,
                            double* __restrict__ part_a, double* __restrict__ part_b) {
  const int64_t total = (int64_t)bd * bd;
  const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  double qa = 0.0, qb = 0.0;
  if (idx < total) {
    const double a = nA[idx], b = nB[idx];
    sA[idx] = make_screen(a);
    const int64_t k = idx / bd, j = idx % bd;
    sBT[j * bd + k] = make_screen(b);
    qa = a * a;
    qb = b * b;
  }
  for (int off = 16; off > 0; off >>= 1) {
    qa += __shfl_xor_sync(0xffffffffu, qa, off);
    qb += __shfl_xor_sync(0xffffffffu, qb, off);
  }
  __shared__ double wa[8], wb[8];
  if ((threadIdx.x & 31) == 0) {
    wa[threadIdx.x / 32] = qa;
    wb[threadIdx.x / 32] = qb;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double sa = 0.0, sb = 0.0;
    for (int w = 0; w < (int)(blockDim.x / 32); ++w) {
      sa += wa[w];
      sb += wb[w];
    }
    part_a[blockIdx.x] = sa;
    part_b[blockIdx.x] = sb;
  }
}

__global__ void norms_kernel(const double* __restrict__ part_a, const double* __restrict__ part_b,
                             int nparts, PlanDevice* __restrict__ pd) {
  __shared__ double sa[256], sb[256];
  double a = 0.0, b = 0.0;
  for (int i = threadIdx.x; i < nparts; i += blockDim.x) {
    a += part_a[i];
    b += part_b[i];
  }
  sa[threadIdx.x] = a;
  sb[threadIdx.x] = b;
  __syncthreads();
  for (int s = blockDim.x / 2; s > 0; s >>= 1) {
    if ((int)threadIdx.x < s) {
      sa[threadIdx.x] += sa[threadIdx.x + s];
      sb[threadIdx.x] += sb[threadIdx.x + s];
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    const double na = sqrt(sa[0]), nb = sqrt(sb[0]);
    pd->norm_a = na;
    pd->norm_b = nb;
    const double ab = na * nb;
    pd->inv_ab = ab > 0.0 ? 1.0 / ab : 0.0;
  }
  for (int i = threadIdx.x; i < kFlagBins; i += blockDim.x) {
    pd->bin_sum[i] = 0.0;
    pd->bin_cnt[i] = 0;
  }
}

struct CountParts {
  long long* S;
  int* kmax;
  int* nonempty;
  double* b1;
  double* b2sq;
};

__global__ void __launch_bounds__(kWarpsPerCta * 32)
    count_kernel(const Screen* __restrict__ sA, const Screen* __restrict__ sBT,
                 const double* __restrict__ nA, const double* __restrict__ nB, int bd,
                 TauScreen T, int split, PlanDevice* __restrict__ pd, int* __restrict__ cnt,
                 CountParts parts, uint8_t* __restrict__ needA, uint8_t* __restrict__ needB) {
  __shared__ double s_bin_sum[kFlagBins];
  __shared__ int s_bin_cnt[kFlagBins];
  __shared__ long long s_S[kWarpsPerCta];
  __shared__ int s_kmax[kWarpsPerCta], s_ne[kWarpsPerCta];
  __shared__ double s_b1[kWarpsPerCta], s_b2[kWarpsPerCta];
  if (split) {
    for (int i = threadIdx.x; i < kFlagBins; i += blockDim.x) {
      s_bin_sum[i] = 0.0;
      s_bin_cnt[i] = 0;
    }
    __syncthreads();
  }
  const int warp = threadIdx.x / 32, lane = threadIdx.x & 31;
  const int64_t t = (int64_t)blockIdx.x * kWarpsPerCta + warp;
  const int64_t tiles = (int64_t)bd * bd;
  int count = 0;
  double skipped = 0.0;
  if (t < tiles) {
    const int i = (int)(t / bd), j = (int)(t % bd);
    const Screen* ra = sA + (int64_t)i * bd;
    const Screen* rb = sBT + (int64_t)j * bd;
    const double inv = pd->inv_ab;
    int inv_e;
    const float inv_m = (float)frexp(inv, &inv_e);
    ExtSum sk{0.0f, 0};  // skipped relative products
    int run_bin = kFlagBinMin - 1, run_cnt = 0;
    double run_sum = 0.0;
    for (int k0 = 0; k0 < bd; k0 += 32) {
      const int k = k0 + lane;
      bool s = false;
      Screen a{}, b{};
      if (k < bd) {
        a = ra[k];
        b = rb[k];
        s = survives(a, b, nA + (int64_t)i * bd + k, nB + (int64_t)k * bd + j, T);
        if (!s) {
          ext_add_rel(sk, a, b, inv_m, inv_e);
        } else if (split) {
          const double p = __dmul_rn(nA[(int64_t)i * bd + k], nB[(int64_t)k * bd + j]);
          const int bin = rel_bin(p, inv);
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
    skipped = ext_value(ext_warp_sum(sk));
    if (lane == 0) {
      cnt[t] = count;
      needA[t] = 0;   // the fill kernel sets the blocks survivors use
      needB[t] = 0;
    }
  }
  if (lane == 0) {
    s_S[warp] = t < tiles ? count : 0;
    s_kmax[warp] = t < tiles ? count : 0;
    s_ne[warp] = (t < tiles && count > 0) ? 1 : 0;
    s_b1[warp] = t < tiles ? skipped : 0.0;
    s_b2[warp] = t < tiles ? skipped * skipped : 0.0;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    long long S = 0;
    int km = 0, ne = 0;
    double b1 = 0.0, b2 = 0.0;
    for (int w = 0; w < kWarpsPerCta; ++w) {
      S += s_S[w];
      km = max(km, s_kmax[w]);
      ne += s_ne[w];
      b1 += s_b1[w];
      b2 += s_b2[w];
    }
    parts.S[blockIdx.x] = S;
    parts.kmax[blockIdx.x] = km;
    parts.nonempty[blockIdx.x] = ne;
    parts.b1[blockIdx.x] = b1;
    parts.b2sq[blockIdx.x] = b2;
  }
  if (split) {
    __syncthreads();
    for (int i = threadIdx.x; i < kFlagBins; i += blockDim.x) {
      if (s_bin_cnt[i]) {
        atomicAdd(&pd->bin_sum[i], s_bin_sum[i]);
        atomicAdd(&pd->bin_cnt[i], (unsigned long long)s_bin_cnt[i]);
      }
    }
  }
}

constexpr int kFinThreads = 1024;

__global__ void __launch_bounds__(kFinThreads)
    finalize_kernel(const int* __restrict__ cnt, int bd, CountParts parts, int nparts, int split,
                    double c1, double target_rel, PlanDevice* __restrict__ pd,
                    int* __restrict__ tile_ptr, int* __restrict__ order) {
  __shared__ long long s_ll[kFinThreads];
  __shared__ double s_d1[kFinThreads], s_d2[kFinThreads];
  __shared__ int s_i1[kFinThreads], s_i2[kFinThreads];
  __shared__ int s_hist[kMaxBd + 1];
  const int tid = threadIdx.x;
  const int64_t tiles = (int64_t)bd * bd;

  // 1. statistics from the count kernel's per-CTA parts
  long long S = 0;
  int km = 0, ne = 0;
  double b1 = 0.0, b2 = 0.0;
  for (int p = tid; p < nparts; p += kFinThreads) {
    S += parts.S[p];
    km = max(km, parts.kmax[p]);
    ne += parts.nonempty[p];
    b1 += parts.b1[p];
    b2 += parts.b2sq[p];
  }
  s_ll[tid] = S;
  s_i1[tid] = km;
  s_i2[tid] = ne;
  s_d1[tid] = b1;
  s_d2[tid] = b2;
  for (int i = tid; i <= bd; i += kFinThreads) s_hist[i] = 0;
  __syncthreads();
  for (int s = kFinThreads / 2; s > 0; s >>= 1) {
    if (tid < s) {
      s_ll[tid] += s_ll[tid + s];
      s_i1[tid] = max(s_i1[tid], s_i1[tid + s]);
      s_i2[tid] += s_i2[tid + s];
      s_d1[tid] += s_d1[tid + s];
      s_d2[tid] += s_d2[tid + s];
    }
    __syncthreads();
  }
  if (tid == 0) {
    const double ab = pd->norm_a * pd->norm_b;
    pd->survivors = s_ll[0];
    pd->max_tile = s_i1[0];
    pd->nonempty = s_i2[0];
    pd->bound1 = s_d1[0] * ab;
    pd->bound2 = sqrt(s_d2[0]) * ab;
    pd->valid_ratio = (double)s_ll[0] / ((double)bd * (double)bd * (double)bd);
    // split flag binade: largest m with c1 * sum_{bin < m} p <= budget
    int m = kFlagBinMin - 1;
    long long flagged = 0;
    if (split) {
      const double budget = 0.5 * (target_rel * ab - pd->bound2);
      if (budget >= 0.0) {
        double below = 0.0;
        for (int mm = kFlagBinMin - 1; mm <= 1; ++mm) {
          // below = sum over bins < mm
          if (mm - 1 >= kFlagBinMin) below += pd->bin_sum[mm - 1 - kFlagBinMin];
          if (c1 * below <= budget) m = mm;
        }
      }
      for (int b = kFlagBinMin; b <= 1; ++b)
        if (b >= m) flagged += (long long)pd->bin_cnt[b - kFlagBinMin];
    }
    pd->flag_exp = m;
    pd->flagged = flagged;
  }
  __syncthreads();

  // 2. exclusive scan of per-tile counts -> tile_ptr (chunk per thread)
  const int64_t chunk = (tiles + kFinThreads - 1) / kFinThreads;
  const int64_t c0 = min(tiles, chunk * tid), c1e = min(tiles, c0 + chunk);
  long long local = 0;
  for (int64_t t = c0; t < c1e; ++t) {
    const int c = cnt[t];
    local += c;
    atomicAdd(&s_hist[c], 1);
  }
  s_ll[tid] = local;
  __syncthreads();
  for (int off = 1; off < kFinThreads; off <<= 1) {   // Hillis-Steele inclusive scan
    long long v = tid >= off ? s_ll[tid - off] : 0;
    __syncthreads();
    s_ll[tid] += v;
    __syncthreads();
  }
  long long run = s_ll[tid] - local;
  for (int64_t t = c0; t < c1e; ++t) {
    tile_ptr[t] = (int)run;
    run += cnt[t];
  }
  if (tid == kFinThreads - 1) tile_ptr[tiles] = (int)s_ll[kFinThreads - 1];
  __syncthreads();

  // 3. longest-first order: bucket offsets in decreasing count
  if (tid == 0) {
    int acc = 0;
    for (int c = bd; c >= 0; --c) {
      const int h = s_hist[c];
      s_hist[c] = acc;
      acc += h;
    }
  }
  __syncthreads();
  for (int64_t t = c0; t < c1e; ++t) {
    const int pos = atomicAdd(&s_hist[cnt[t]], 1);
    order[pos] = (int)t;
  }
}

__global__ void __launch_bounds__(kWarpsPerCta * 32)
    fill_kernel(const Screen* __restrict__ sA, const Screen* __restrict__ sBT,
                const double* __restrict__ nA, const double* __restrict__ nB, int bd, TauScreen T,
                int split, const PlanDevice* __restrict__ pd, const int* __restrict__ cnt,
                const int* __restrict__ tile_ptr, uint16_t* __restrict__ k_idx,
                uint8_t* __restrict__ needA, uint8_t* __restrict__ needB) {
  const int warp = threadIdx.x / 32, lane = threadIdx.x & 31;
  const int64_t t = (int64_t)blockIdx.x * kWarpsPerCta + warp;
  if (t >= (int64_t)bd * bd) return;
  if (cnt[t] == 0) return;
  const int i = (int)(t / bd), j = (int)(t % bd);
  const Screen* ra = sA + (int64_t)i * bd;
  const Screen* rb = sBT + (int64_t)j * bd;
  const double inv = pd->inv_ab;
  const int m = pd->flag_exp;
  int base = tile_ptr[t];
  for (int k0 = 0; k0 < bd; k0 += 32) {
    const int k = k0 + lane;
    bool s = false;
    if (k < bd) s = survives(ra[k], rb[k], nA + (int64_t)i * bd + k, nB + (int64_t)k * bd + j, T);
    const unsigned ball = __ballot_sync(0xffffffffu, s);
    if (s) {
      uint16_t v = (uint16_t)k;
      if (split) {
        const double p = __dmul_rn(nA[(int64_t)i * bd + k], nB[(int64_t)k * bd + j]);
        if (rel_bin(p, inv) >= m) v |= kSplitFlag;
      }
      k_idx[base + __popc(ball & ((1u << lane) - 1u))] = v;
      needA[(int64_t)i * bd + k] = 1;   // benign: every writer stores 1
      needB[(int64_t)k * bd + j] = 1;
    }
    base += __popc(ball);
  }
}

}  // namespace

cudaError_t run_plan(PlanBuffers& b, const double* nA, const double* nB, double tau,
                     double target_rel, int split, double c1, cudaStream_t s) {
  const int bd = b.bd;
  const int64_t tiles = (int64_t)bd * bd;
  const int prep_ctas = (int)((tiles + 255) / 256);
  prep_kernel<<<prep_ctas, 256, 0, s>>>(nA, nB, bd, b.sA, b.sBT, b.part_a, b.part_b);
  norms_kernel<<<1, 256, 0, s>>>(b.part_a, b.part_b, prep_ctas, b.pd);
  const TauScreen T = make_tau_screen(tau);
  const int count_ctas = (int)((tiles + kWarpsPerCta - 1) / kWarpsPerCta);
  CountParts parts{b.part_S, b.part_kmax, b.part_ne, b.part_b1, b.part_b2};
  count_kernel<<<count_ctas, kWarpsPerCta * 32, 0, s>>>(b.sA, b.sBT, nA, nB, bd, T, split, b.pd,
                                                        b.cnt, parts, b.needA, b.needB);
  finalize_kernel<<<1, kFinThreads, 0, s>>>(b.cnt, bd, parts, count_ctas, split, c1, target_rel,
                                            b.pd, b.tile_ptr, b.order);
  fill_kernel<<<count_ctas, kWarpsPerCta * 32, 0, s>>>(b.sA, b.sBT, nA, nB, bd, T, split, b.pd,
                                                       b.cnt, b.tile_ptr, b.k_idx, b.needA,
                                                       b.needB);
  return cudaPeekAtLastError();
}

int64_t plan_part_count(int bd) {
  const int64_t tiles = (int64_t)bd * bd;
  return std::max<int64_t>((tiles + 255) / 256, (tiles + kWarpsPerCta - 1) / kWarpsPerCta);
}

}  // namespace spamm
