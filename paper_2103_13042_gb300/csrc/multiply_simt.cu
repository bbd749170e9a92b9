// Plain FP32 multiply on the SIMT cores (Section 3.3's FP32 multiplication
// kernel; the baseline the tensor-core modes are measured against).
//
// Persistent CTAs walk the non-empty tiles of all instances (most survivors
// first) with a grid stride; the caller writes the empty tiles with the
// coalesced zero-fill kernel.  A non-empty tile (i, j) streams its
// surviving k in 32-wide slices of the inner dimension: the A slice
// A[i, k][:, s:s+32] is stored transposed and the B slice B[k, j][s:s+32, :]
// as is, both in shared memory, double buffered through registers so the next
// slice's global loads overlap the current slice's FMAs.  Each of the 256
// threads keeps a (leaf/16) x (leaf/16) register tile of C and accumulates
// in FP32 FMA over every surviving k.  Empty tiles are written as zeros with
// coalesced float4 stores (beta = 0) by that kernel.
#include "tc_common.cuh"

namespace spamm {
namespace {

constexpr int kThreads = 256;
constexpr int kSlice = 32;

template <int LEAF>
struct SimtTile {
  static constexpr int TM = LEAF / 16;                    // C rows (and cols) per thread
  static constexpr int kLoadsA = LEAF * kSlice / 4 / kThreads;  // float4 per thread per slice
};

// Loads 4 consecutive floats of row r, columns c..c+3 of a rows x cols matrix
// with leading dimension ld, zero outside it.
__device__ __forceinline__ float4 load4(const float* __restrict__ M, int64_t rows, int64_t cols,
                                        int64_t ld, int64_t r, int64_t c, bool vec) {
  if (r >= rows) return make_float4(0.f, 0.f, 0.f, 0.f);
  const float* p = M + r * ld + c;
  if (vec && c + 3 < cols) return __ldg(reinterpret_cast<const float4*>(p));
  float4 v;
  v.x = c < cols ? __ldg(p) : 0.f;
  v.y = c + 1 < cols ? __ldg(p + 1) : 0.f;
  v.z = c + 2 < cols ? __ldg(p + 2) : 0.f;
  v.w = c + 3 < cols ? __ldg(p + 3) : 0.f;
  return v;
}

// TM consecutive floats from 16-byte (TM >= 4) or 8-byte (TM = 2) aligned shared memory.
template <int TM>
__device__ __forceinline__ void read_row(const float* p, float* out) {
  if constexpr (TM >= 4) {
#pragma unroll
    for (int v = 0; v < TM; v += 4) {
      const float4 x = *reinterpret_cast<const float4*>(p + v);
      out[v] = x.x; out[v + 1] = x.y; out[v + 2] = x.z; out[v + 3] = x.w;
    }
  } else {
    const float2 x = *reinterpret_cast<const float2*>(p);
    out[0] = x.x; out[1] = x.y;
  }
}

template <int TM>
__device__ __forceinline__ void write_row(float* p, const float* v) {
  if constexpr (TM >= 4) {
#pragma unroll
    for (int q = 0; q < TM; q += 4)
      *reinterpret_cast<float4*>(p + q) = make_float4(v[q], v[q + 1], v[q + 2], v[q + 3]);
  } else {
    *reinterpret_cast<float2*>(p) = make_float2(v[0], v[1]);
  }
}

template <int LEAF>
__global__ void __launch_bounds__(kThreads) simt_kernel(InstRef R, PlanBuffers Bf, int dynamic) {
  pdl_wait();
  using T = SimtTile<LEAF>;
  constexpr int TM = T::TM;
  constexpr int kLoads = T::kLoadsA;
  // A slice transposed: sA[buf][s][r] (r = row within the leaf), B slice sB[buf][s][c]
  extern __shared__ __align__(16) float smem[];
  float (*sA)[kSlice][LEAF + 4] = reinterpret_cast<float (*)[kSlice][LEAF + 4]>(smem);
  float (*sB)[kSlice][LEAF + 4] =
      reinterpret_cast<float (*)[kSlice][LEAF + 4]>(smem + 2 * kSlice * (LEAF + 4));

  const int tid = threadIdx.x;
  const int tx = tid % 16, ty = tid / 16;
  const int64_t ne = Bf.bdev->nonempty;   // empty tiles are zero-filled by another kernel

  __shared__ int s_next;
  for (int64_t w = blockIdx.x;; w += gridDim.x) {
    if (dynamic) {   // next tile from the global counter (its use ends at the loop's barrier)
      if (tid == 0) s_next = atomicAdd(&Bf.bdev->mul_ticket, 1);
      __syncthreads();
      w = s_next;
    }
    if (w >= ne) break;
    const int g = Bf.order[w];
    const Inst& in = R.at(inst_of(R, Bf, g));
    const int bn = in.bn;
    const int64_t m = in.m, kd = in.kd, n = in.n;
    const int64_t lda = in.lda, ldb = in.ldb, ldc = in.ldc;
    const float* __restrict__ A = in.A;
    const float* __restrict__ B = in.B;
    float* __restrict__ C = in.C;
    const bool vec_a = (lda % 4) == 0, vec_b = (ldb % 4) == 0, vec_c = (ldc % 4) == 0;
    const uint16_t* __restrict__ k_idx = Bf.k_idx;
    const int64_t t = g - in.tile0;
    const int i = (int)(t / bn), j = (int)(t % bn);
    const int beg = Bf.tile_beg[g], end = beg + Bf.cnt[g];
    const int64_t r0 = (int64_t)i * LEAF, c0 = (int64_t)j * LEAF;

    float acc[TM][TM];
#pragma unroll
    for (int a = 0; a < TM; ++a)
#pragma unroll
      for (int b = 0; b < TM; ++b) acc[a][b] = 0.f;

    const int nslices = (end - beg) * (LEAF / kSlice);
    float4 ra[kLoads], rb[kLoads];

    // slice q -> (k, s0): A rows r0.., cols k*LEAF + s0..; B rows k*LEAF + s0.., cols c0..
    auto fetch = [&](int q) {
      const int k = k_idx[beg + q / (LEAF / kSlice)] & 0x3ff;
      const int s0 = (q % (LEAF / kSlice)) * kSlice;
#pragma unroll
      for (int l = 0; l < kLoads; ++l) {
        const int e = (tid + l * kThreads) * 4;      // element index in the slice
        // A slice: LEAF rows x 32 cols, float4 along the columns
        const int ar = e / kSlice, ac = e % kSlice;
        ra[l] = load4(A, m, kd, lda, r0 + ar, (int64_t)k * LEAF + s0 + ac, vec_a);
        // B slice: 32 rows x LEAF cols, float4 along the columns
        const int br = e / LEAF, bc = e % LEAF;
        rb[l] = load4(B, kd, n, ldb, (int64_t)k * LEAF + s0 + br, c0 + bc, vec_b);
      }
    };
    auto stash = [&](int buf) {
#pragma unroll
      for (int l = 0; l < kLoads; ++l) {
        const int e = (tid + l * kThreads) * 4;
        const int ar = e / kSlice, ac = e % kSlice;
        sA[buf][ac + 0][ar] = ra[l].x;
        sA[buf][ac + 1][ar] = ra[l].y;
        sA[buf][ac + 2][ar] = ra[l].z;
        sA[buf][ac + 3][ar] = ra[l].w;
        const int br = e / LEAF, bc = e % LEAF;
        *reinterpret_cast<float4*>(&sB[buf][br][bc]) = rb[l];
      }
    };

    fetch(0);
    __syncthreads();  // previous tile's readers are done with both buffers
    stash(0);
    __syncthreads();
    for (int q = 0; q < nslices; ++q) {
      const int buf = q & 1;
      if (q + 1 < nslices) fetch(q + 1);
#pragma unroll 8
      for (int s = 0; s < kSlice; ++s) {
        float a[TM], b[TM];
        read_row<TM>(&sA[buf][s][ty * TM], a);
        read_row<TM>(&sB[buf][s][tx * TM], b);
#pragma unroll
        for (int u = 0; u < TM; ++u)
#pragma unroll
          for (int v = 0; v < TM; ++v) acc[u][v] = __fmaf_rn(a[u], b[v], acc[u][v]);
      }
      if (q + 1 < nslices) stash(buf ^ 1);
      __syncthreads();
    }

    // epilogue: C = alpha * acc + beta * C (the old C is read only when beta != 0)
    const float alpha = in.alpha, beta = in.beta;
#pragma unroll
    for (int u = 0; u < TM; ++u) {
      const int64_t r = r0 + ty * TM + u;
      const int64_t c = c0 + tx * TM;
      float* p = C + r * ldc + c;
      const bool row_in = r < m;
      if (beta != 0.0f && row_in) {
#pragma unroll
        for (int q = 0; q < TM; ++q)
          acc[u][q] = c + q < n ? __fmaf_rn(beta, p[q], __fmul_rn(alpha, acc[u][q])) : 0.0f;
      } else {
#pragma unroll
        for (int q = 0; q < TM; ++q) acc[u][q] = __fmul_rn(alpha, acc[u][q]);
      }
      if (!row_in) continue;
      if (vec_c && c + TM - 1 < n) {
        write_row<TM>(p, acc[u]);
      } else {
#pragma unroll
        for (int q = 0; q < TM; ++q)
          if (c + q < n) p[q] = acc[u][q];
      }
    }
    if (in.nC) {   // C's norm map for a chained product: the tile's stored values
      float v[TM * TM];
#pragma unroll
      for (int u = 0; u < TM; ++u)
#pragma unroll
        for (int q = 0; q < TM; ++q) {
          const bool inside = r0 + ty * TM + u < m && c0 + tx * TM + q < n;
          v[u * TM + q] = inside ? acc[u][q] : 0.0f;
        }
      SumSq ss = sumsq_empty();
      sumsq_group<TM * TM>(ss, v);
#pragma unroll
      for (int off = 16; off > 0; off >>= 1) {
        const float h = __shfl_xor_sync(0xffffffffu, ss.hi, off);
        const float l = __shfl_xor_sync(0xffffffffu, ss.lo, off);
        const int e = __shfl_xor_sync(0xffffffffu, ss.e, off);
        sumsq_merge_any(ss, h, l, e);
      }
      __shared__ SumSq s_norm[kThreads / 32];
      if ((tid & 31) == 0) s_norm[tid / 32] = ss;
      __syncthreads();
      if (tid == 0) {
        SumSq tot = s_norm[0];
        for (int w = 1; w < kThreads / 32; ++w) sumsq_merge_any(tot, s_norm[w].hi, s_norm[w].lo, s_norm[w].e);
        in.nC[t] = sumsq_sqrt(tot);
      }
    }
  }
}

template <int LEAF>
cudaError_t launch(const InstRef& ref, const PlanBuffers& b, int schedule, cudaStream_t s) {
  constexpr size_t smem = 4 * kSlice * (LEAF + 4) * sizeof(float);
  int dev = 0, sms = 0, per_sm = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  cudaFuncSetAttribute(simt_kernel<LEAF>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, simt_kernel<LEAF>, kThreads, smem);
  const int grid = (int)std::max<int64_t>(
      1, std::min<int64_t>(b.tiles, (int64_t)sms * std::max(1, per_sm)));
  cudaError_t e = launch_pdl(simt_kernel<LEAF>, dim3(grid), dim3(kThreads), smem, s, ref, b,
                             (int)(schedule == kScheduleDynamic));
  if (e != cudaSuccess) return e;
  return cudaPeekAtLastError();
}

}  // namespace

cudaError_t launch_multiply_simt(const InstRef& ref, const PlanBuffers& b, int leaf,
                                 int schedule, cudaStream_t s) {
  switch (leaf) {
    case 32: return launch<32>(ref, b, schedule, s);
    case 64: return launch<64>(ref, b, schedule, s);
    case 128: return launch<128>(ref, b, schedule, s);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace spamm
