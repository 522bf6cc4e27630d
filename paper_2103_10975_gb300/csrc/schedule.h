// Batch schedule (host code): see schedule.cu.
#pragma once
#include <vector>

namespace mlg {

// Cost estimate of one system of side n (dim 2 or 3): N * n^2.
double system_cost(int dim, int n);

// Splits `ctas` CTAs into groups and assigns each of the `count` systems to a
// group.  Returns the number of groups G; group_ctas[0..G-1] sum to at most
// `ctas`; group_of[i] is system i's group; order lists the systems by
// decreasing cost (the order in which each group takes its systems).
int plan_batch(int dim, int count, const int* n, int ctas, std::vector<int>& group_ctas,
               std::vector<int>& group_of, std::vector<int>& order);

}  // namespace mlg
