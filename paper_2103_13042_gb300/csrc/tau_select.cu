// Choosing tau for a target error: the arbiter of the learned tau and its
// fallback.  The paper chooses tau by a search for a valid ratio (Section
// 3.5.2); here tau is chosen for the pruning error itself,
//
//     e(tau) = ||AB - SpAMM(A, B, tau)||_F / (||A||_F ||B||_F)     (Eq. 5 error),
//
// measured without forming AB:
//  1. certify: tau_ref = the largest tau on a log10 grid of [1e-60, 1] ||A|| ||B||
//     (36 bisection steps of the exponent) whose skipped-product bound
//     bound2(tau_ref) <= ref_rel ||A|| ||B||.  Then ||AB - SpAMM(tau_ref)||_F is
//     at most ref_rel ||A|| ||B||.
//  2. error: for tau > tau_ref, AB - SpAMM(tau) = C_band + (AB - SpAMM(tau_ref))
//     with C_band the product over the band tau_ref <= p < tau, so e(tau) is
//     ||C_band||_F / (||A|| ||B||) to within ref_rel.  C_band is one band plan,
//     one FP32 multiply into caller scratch and one Frobenius reduction.
//  3. select: the network's tau (spamm_tau_predict) checked once; on a miss, or
//     without a network, bisection on e: bracket [lo, hi] from tau0 =
//     target ||A|| ||B|| by factors of 10 (up while e(hi) <= target, or down
//     until an admissible tau appears), then geometric bisection until
//     hi / lo <= 1.01 or 40 evaluations; the largest tested admissible tau.
#include <cmath>

#include "engine.cuh"

using namespace spamm;

namespace {

constexpr int kCertifySteps = 36;
constexpr double kCertifyLo = -60.0;   // log10 of the smallest relative tau tried
constexpr int kBisectMaxEvals = 40;
constexpr double kBisectRatio = 1.01;

spamm_status_t cuda_fail() {
  (void)cudaGetLastError();
  return SPAMM_ERR_CUDA;
}

bool aligned16(const void* p) { return (reinterpret_cast<uintptr_t>(p) & 15u) == 0; }

// The counting half of a plan at tau; the statistics to *out (blocks).
spamm_status_t count_stats(Engine& e, const double* nA, const double* nB, double tau,
                           cudaStream_t s, PlanDevice* out) {
  Inst& in = e.insts[0];
  in.nA = nA;
  in.nB = nB;
  in.T = make_tau_screen(tau);
  in.band = 0;
  in.split = 0;
  in.quant = 0;
  if (run_plan_count(make_ref(e.insts.data(), nullptr, 1), e.buf, s) != cudaSuccess)
    return cuda_fail();
  SPAMM_CUDA_TRY(cudaMemcpyAsync(out, e.buf.pd, sizeof(PlanDevice), cudaMemcpyDeviceToHost, s));
  SPAMM_CUDA_TRY(cudaStreamSynchronize(s));
  return SPAMM_OK;
}

spamm_status_t certify(Engine& e, const double* nA, const double* nB, double ref_rel,
                       cudaStream_t s, double* tau_ref, double* ab_out) {
  PlanDevice h;
  spamm_status_t st = count_stats(e, nA, nB, 0.0, s, &h);
  if (st != SPAMM_OK) return st;
  const double ab = h.norm_a * h.norm_b;
  *ab_out = ab;
  if (!(ab > 0.0) || std::isinf(ab)) {   // a zero (or non-finite) operand: nothing to certify
    *tau_ref = 0.0;
    return SPAMM_OK;
  }
  double lo = kCertifyLo, hi = 0.0;
  for (int it = 0; it < kCertifySteps; ++it) {
    const double mid = 0.5 * (lo + hi);
    st = count_stats(e, nA, nB, ab * std::pow(10.0, mid), s, &h);
    if (st != SPAMM_OK) return st;
    if (h.bound2 <= ref_rel * ab) lo = mid;
    else hi = mid;
  }
  *tau_ref = ab * std::pow(10.0, lo);
  return SPAMM_OK;
}

// e(tau) relative to ||A|| ||B|| (0 at or below tau_ref).
spamm_status_t band_error(Engine& e, const double* nA, const double* nB, const float* A,
                          const float* B, float* scratch, int64_t n, double tau, double tau_ref,
                          double ab, cudaStream_t s, double* err) {
  if (!(tau > tau_ref) || !(ab > 0.0)) {
    *err = 0.0;
    return SPAMM_OK;
  }
  Inst& in = e.insts[0];
  in.nA = nA;
  in.nB = nB;
  in.A = A;
  in.B = B;
  in.C = scratch;
  in.lda = in.ldb = in.ldc = in.n;
  in.alpha = 1.0f;
  in.beta = 0.0f;
  in.nC = nullptr;
  in.T = make_tau_screen(tau_ref);
  in.T_hi = make_tau_screen(tau);
  in.band = 1;
  in.split = 0;
  in.quant = 0;
  const InstRef ref = make_ref(e.insts.data(), nullptr, 1);
  cudaError_t ce = run_plan(ref, e.buf, s);
  in.band = 0;
  if (ce == cudaSuccess) ce = launch_multiply_simt(ref, e.buf, e.leaf, kScheduleStatic, s);
  if (ce == cudaSuccess) ce = launch_zero_empty_tiles(ref, e.buf, e.leaf, s);
  if (ce != cudaSuccess) return cuda_fail();
  double norm = 0.0;
  const spamm_status_t st = spamm_frobenius_diff(scratch, nullptr, n * n, &norm, s);
  if (st != SPAMM_OK) return st;
  *err = norm / ab;
  return SPAMM_OK;
}

spamm_status_t check_common(spamm_plan_t plan, const double* nA, const double* nB) {
  if (!plan || !nA || !nB) return SPAMM_ERR_INVALID_ARG;
  if (plan->general) return SPAMM_ERR_UNSUPPORTED;   // square plans only
  if (!aligned16(nA) || !aligned16(nB)) return SPAMM_ERR_INVALID_ARG;
  return SPAMM_OK;
}

spamm_status_t check_operands(const float* A, const float* B, const float* scratch) {
  if (!A || !B || !scratch) return SPAMM_ERR_INVALID_ARG;
  if (!aligned16(A) || !aligned16(B) || !aligned16(scratch)) return SPAMM_ERR_INVALID_ARG;
  if (scratch == A || scratch == B) return SPAMM_ERR_INVALID_ARG;
  return SPAMM_OK;
}

}  // namespace

extern "C" {

spamm_status_t spamm_tau_certify(spamm_plan_t plan, const double* normA, const double* normB,
                                 double ref_rel, double* tau_ref, double* norm_ab, void* stream) {
  spamm_status_t st = check_common(plan, normA, normB);
  if (st != SPAMM_OK) return st;
  if (!tau_ref || !(ref_rel > 0.0) || std::isinf(ref_rel)) return SPAMM_ERR_INVALID_ARG;
  double ab = 0.0;
  st = certify(plan->eng, normA, normB, ref_rel, (cudaStream_t)stream, tau_ref, &ab);
  if (st == SPAMM_OK && norm_ab) *norm_ab = ab;
  return st;
}

spamm_status_t spamm_tau_error(spamm_plan_t plan, const double* normA, const double* normB,
                               const float* A, const float* B, double tau, double tau_ref,
                               float* scratch, double* err, void* stream) {
  spamm_status_t st = check_common(plan, normA, normB);
  if (st != SPAMM_OK) return st;
  st = check_operands(A, B, scratch);
  if (st != SPAMM_OK) return st;
  if (!err || std::isnan(tau) || tau < 0.0 || std::isnan(tau_ref) || tau_ref < 0.0)
    return SPAMM_ERR_INVALID_ARG;
  const cudaStream_t s = (cudaStream_t)stream;
  PlanDevice h;
  st = count_stats(plan->eng, normA, normB, 0.0, s, &h);   // ||A||, ||B|| from the norm maps
  if (st != SPAMM_OK) return st;
  return band_error(plan->eng, normA, normB, A, B, scratch, plan->n, tau, tau_ref,
                    h.norm_a * h.norm_b, s, err);
}

spamm_status_t spamm_tau_select(spamm_plan_t plan, const double* normA, const double* normB,
                                const float* A, const float* B, double target_rel_err,
                                const float* weights, float* scratch, double* tau,
                                int32_t* evals, double* achieved, void* stream) {
  spamm_status_t st = check_common(plan, normA, normB);
  if (st != SPAMM_OK) return st;
  st = check_operands(A, B, scratch);
  if (st != SPAMM_OK) return st;
  if (!tau || !(target_rel_err > 0.0) || std::isinf(target_rel_err)) return SPAMM_ERR_INVALID_ARG;
  const cudaStream_t s = (cudaStream_t)stream;
  Engine& e = plan->eng;
  const double eps = target_rel_err;
  double tau_ref = 0.0, ab = 0.0;
  st = certify(e, normA, normB, 1e-11, s, &tau_ref, &ab);
  if (st != SPAMM_OK) return st;
  int n_eval = 0;
  double last_err = 0.0;
  auto err_at = [&](double t, double* out) -> spamm_status_t {
    ++n_eval;
    return band_error(e, normA, normB, A, B, scratch, plan->n, t, tau_ref, ab, s, out);
  };
  auto finish = [&](double t, double et) {
    *tau = t;
    if (evals) *evals = n_eval;
    if (achieved) *achieved = et;
    return SPAMM_OK;
  };
  if (!(ab > 0.0) || std::isinf(ab)) return finish(0.0, 0.0);   // nothing to prune safely

  // the network's tau, checked once
  if (weights) {
    double tp = 0.0;
    st = spamm_tau_predict(plan, normA, normB, eps, weights, &tp, stream);
    if (st != SPAMM_OK) return st;
    double ep = 0.0;
    st = err_at(tp, &ep);
    if (st != SPAMM_OK) return st;
    if (ep <= eps) return finish(tp, ep);
  }
  // bisection on e (the fallback, and the arbiter of the network's answer)
  const int first = n_eval;
  auto used = [&]() { return n_eval - first; };
  double lo_err = 0.0;
  auto ok = [&](double t, bool* res) -> spamm_status_t {
    double et = 0.0;
    const spamm_status_t r = err_at(t, &et);
    if (r != SPAMM_OK) return r;
    *res = et <= eps;
    last_err = et;
    return SPAMM_OK;
  };
  double lo = 0.0, hi = eps * ab;
  bool good = false;
  if ((st = ok(hi, &good)) != SPAMM_OK) return st;
  if (good) {
    lo = hi;
    lo_err = last_err;
    hi *= 10.0;
    while (used() < kBisectMaxEvals) {
      if ((st = ok(hi, &good)) != SPAMM_OK) return st;
      if (!good) break;
      lo = hi;
      lo_err = last_err;
      hi *= 10.0;
    }
    if (used() >= kBisectMaxEvals) return finish(lo, lo_err);
  } else {
    double t = hi / 10.0;
    while (used() < kBisectMaxEvals && t > 0.0) {
      if ((st = ok(t, &good)) != SPAMM_OK) return st;
      if (good) {
        lo = t;
        lo_err = last_err;
        break;
      }
      hi = t;
      t /= 10.0;
    }
    if (lo == 0.0) return finish(0.0, 0.0);
  }
  while (hi / lo > kBisectRatio && used() < kBisectMaxEvals) {
    const double mid = std::sqrt(lo * hi);
    if ((st = ok(mid, &good)) != SPAMM_OK) return st;
    if (good) {
      lo = mid;
      lo_err = last_err;
    } else {
      hi = mid;
    }
  }
  return finish(lo, lo_err);
}

}  // extern "C"
