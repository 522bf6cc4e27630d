// Batch schedule: how the CTAs of one persistent launch are split into groups
// and which systems each group solves (host code only).
//
// The cost of a system is taken as N * n^2: the Arnoldi steps of
// unpreconditioned GMRES on the Poisson operator grow about like n^2 (the
// condition number) and each step moves O(N) values.  Across sides 64..512
// that spans four decades, so a list of one-CTA groups would leave the launch
// waiting for the CTA that drew a 512^2 system.  Systems whose cost exceeds
// the ideal per-CTA load get a group of several CTAs (in proportion, at most
// one per kMinPointsPerCta points); the other CTAs form one-CTA groups; then
// every system not yet placed goes, largest first, to the group on which it
// would finish earliest.
#include <math.h>

#include <algorithm>
#include <numeric>
#include <vector>

#include "../../include/mlgmres.h"
#include "schedule.h"

namespace mlg {

namespace {
constexpr long long kMinPointsPerCta = 512;  // as for single solves
}

double system_cost(int dim, int n) {
  const double N = dim == 2 ? (double)n * n : (double)n * n * n;
  return N * (double)n * (double)n;
}

int plan_batch(int dim, int count, const int* n, int ctas, std::vector<int>& group_ctas,
               std::vector<int>& group_of, std::vector<int>& order) {
  group_ctas.clear();
  group_of.assign(count, -1);
  order.resize(count);
  if (count <= 0 || ctas <= 0) return 0;
  std::vector<double> cost(count);
  double total = 0.0;
  for (int i = 0; i < count; i++) {
    cost[i] = system_cost(dim, n[i]);
    total += cost[i];
  }
  std::iota(order.begin(), order.end(), 0);
  std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return cost[a] > cost[b]; });
  const double ideal = total / ctas;
  std::vector<double> load;
  int left = ctas;
  int placed = 0;
  // dedicated multi-CTA groups for the systems that alone exceed the ideal load
  for (int r = 0; r < count; r++) {
    const int i = order[r];
    const int unplaced_after = count - r - 1;
    int want = (int)ceil(cost[i] / ideal - 1e-9);
    const long long N = dim == 2 ? (long long)n[i] * n[i] : (long long)n[i] * n[i] * n[i];
    const int by_size = (int)std::max<long long>(1, N / kMinPointsPerCta);
    // keep one CTA for the remaining systems
    const int avail = left - (unplaced_after > 0 ? 1 : 0);
    want = std::min(want, std::min(by_size, avail));
    if (want <= 1) break;
    group_ctas.push_back(want);
    load.push_back(cost[i] / want);
    group_of[i] = (int)group_ctas.size() - 1;
    left -= want;
    placed++;
  }
  // one-CTA groups for the rest (no more groups than systems left)
  const int singles = std::min(left, count - placed);
  for (int g = 0; g < singles; g++) {
    group_ctas.push_back(1);
    load.push_back(0.0);
  }
  // LPT: the remaining systems, largest first, to the earliest finish
  for (int r = placed; r < count; r++) {
    const int i = order[r];
    int best = 0;
    double best_t = INFINITY;
    for (int g = 0; g < (int)group_ctas.size(); g++) {
      const double t = load[g] + cost[i] / group_ctas[g];
      if (t < best_t) {
        best_t = t;
        best = g;
      }
    }
    load[best] = best_t;
    group_of[i] = best;
  }
  return (int)group_ctas.size();
}

}  // namespace mlg

extern "C" mlgmres_status mlgmres_batch_plan(int dim, int count, const int* n, int ctas,
                                             int* groups, int* group_ctas, int* group_of) {
  if ((dim != 2 && dim != 3) || count < 1 || ctas < 1 || !n || !groups || !group_ctas ||
      !group_of)
    return MLGMRES_ERR_ARG;
  for (int i = 0; i < count; i++)
    if (n[i] < 1) return MLGMRES_ERR_ARG;
  std::vector<int> gc, gof, order;
  const int G = mlg::plan_batch(dim, count, n, ctas, gc, gof, order);
  *groups = G;
  for (int g = 0; g < G; g++) group_ctas[g] = gc[g];
  for (int i = 0; i < count; i++) group_of[i] = gof[i];
  return MLGMRES_OK;
}
