// How lbm_sw_step(n) maps n time steps to fused launches (host code only; no CUDA
// dependency, so it also compiles into a plain host test program).
#pragma once

#include <algorithm>

namespace lbm {

// Relative cost of one launch of k fused steps (k = 1: one step per launch), measured as
// ms per launch on the 4096^2 FP32 periodic dam-break: 0.253 (one step), 0.291, 0.300,
// 0.309, 0.355, 0.372, 0.577, 0.628 (k = 2 .. 8).  Used only to split the tail of a call
// into launches; every split gives the same bits.
constexpr double kLaunchCost[9] = {0.0, 0.253, 0.291, 0.300, 0.309, 0.355, 0.372, 0.577, 0.628};

constexpr int kMaxTail = 16;  // K + 8 with K <= 8

// Steps per launch for n steps of a handle fusing K (2 .. 8) steps per launch, into plan[]
// (returns the number of launches written, at most max_plan, max_plan > kMaxTail).
// Launches of K while more than K + 8 steps remain, then the cheapest split of the rest
// (at most K + 8 steps) into launches of at most K steps: K itself and even sizes always
// (the two-column kernels), other odd sizes above one only when odd_ok (every side periodic:
// the paired kernel with an even left halo, or the one-column kernel), at most one single
// step.  At K = 6 a call of 20
// steps runs 6 + 6 + 4 + 4, one of 8 runs 4 + 4.  When max_plan runs out first, the
// launches written cover part of n and the caller plans the rest in another call.
inline int plan_launches(int K, bool odd_ok, int n, int* plan, int max_plan) {
  auto allowed = [&](int k) { return k == 1 || k == K || (k < K && (k % 2 == 0 || odd_ok)); };
  int count = 0;
  while (n > K + 8) {
    if (count == max_plan) return count;
    plan[count++] = K;
    n -= K;
  }
  // cheapest split of the remaining n <= K + 8 <= kMaxTail steps
  double best[kMaxTail + 1];
  int first[kMaxTail + 1];
  best[0] = 0.0;
  first[0] = 0;
  for (int m = 1; m <= n; ++m) {
    best[m] = 1e300;
    first[m] = 1;
    for (int k = 1; k <= 8 && k <= m; ++k) {
      if (!allowed(k)) continue;
      const double c = kLaunchCost[k] + best[m - k];
      if (c < best[m]) {
        best[m] = c;
        first[m] = k;
      }
    }
  }
  // larger launches first
  int tail[kMaxTail], nt = 0;
  for (int m = n; m > 0; m -= first[m]) tail[nt++] = first[m];
  std::sort(tail, tail + nt, [](int a, int b) { return a > b; });
  if (count + nt > max_plan) return count;  // the whole tail in the caller's next call
  for (int i = 0; i < nt; ++i) plan[count++] = tail[i];
  return count;
}

}  // namespace lbm
