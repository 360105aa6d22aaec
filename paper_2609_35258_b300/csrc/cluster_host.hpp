// Grouping of cellwise coarsening masks into representative spaces (Sec. 3.2), host side.
//
//  * graded distance of two masks: sum_b |kappa_a(b) - kappa_b(b)| / (3 N_b);
//  * identical masks are merged, the distinct ones ordered by decreasing frequency (equal
//    frequencies by the lexicographic order of the mask); the first seeds cluster 0, every
//    next one joins the nearest centre when that distance is <= tau (the lowest cluster index
//    on equal distances) and otherwise seeds a new cluster; a centre is its seeding mask;
//  * the representative (enclosing) mask is the blockwise minimum over the members.
#pragma once
#include <algorithm>
#include <cstdint>
#include <cstring>
#include <string>
#include <unordered_map>
#include <vector>

namespace mlvs {

struct Clustering {
  std::vector<int> labels;               // per row
  std::vector<std::vector<uint8_t>> reps;  // per cluster, N_b entries
  int n_distinct = 0;
};

inline Clustering cluster_masks(const uint8_t* kappa, long nrow, int nb, double tau) {
  Clustering out;
  out.labels.assign(nrow, 0);
  if (nrow == 0) return out;
  // distinct masks with their counts
  std::unordered_map<std::string, int> idx;
  idx.reserve((size_t)nrow * 2);
  std::vector<int> row_u(nrow);
  std::vector<const uint8_t*> uptr;
  std::vector<long> cnt;
  for (long r = 0; r < nrow; ++r) {
    const uint8_t* p = kappa + (size_t)r * nb;
    std::string key(reinterpret_cast<const char*>(p), nb);
    auto it = idx.find(key);
    if (it == idx.end()) {
      it = idx.emplace(std::move(key), (int)uptr.size()).first;
      uptr.push_back(p);
      cnt.push_back(0);
    }
    ++cnt[it->second];
    row_u[r] = it->second;
  }
  const int nu = (int)uptr.size();
  out.n_distinct = nu;
  std::vector<int> order(nu);
  for (int u = 0; u < nu; ++u) order[u] = u;
  std::sort(order.begin(), order.end(), [&](int a, int b) {
    if (cnt[a] != cnt[b]) return cnt[a] > cnt[b];
    return std::memcmp(uptr[a], uptr[b], nb) < 0;
  });
  std::vector<int> centre;                 // distinct-mask index of every centre
  std::vector<int> ulabel(nu, 0);
  const double denom = 3.0 * nb;
  for (int u : order) {
    if (centre.empty()) {
      centre.push_back(u);
      ulabel[u] = 0;
      continue;
    }
    int best = -1;
    double bd = 0.0;
    for (size_t c = 0; c < centre.size(); ++c) {
      const uint8_t* a = uptr[u];
      const uint8_t* b = uptr[centre[c]];
      long s = 0;
      for (int k = 0; k < nb; ++k) s += std::abs((int)a[k] - (int)b[k]);
      const double d = (double)s / denom;
      if (best < 0 || d < bd) { best = (int)c; bd = d; }
    }
    if (bd <= tau) {
      ulabel[u] = best;
    } else {
      ulabel[u] = (int)centre.size();
      centre.push_back(u);
    }
  }
  out.reps.assign(centre.size(), std::vector<uint8_t>(nb, 255));
  for (int u = 0; u < nu; ++u) {
    auto& rep = out.reps[ulabel[u]];
    const uint8_t* p = uptr[u];
    for (int k = 0; k < nb; ++k) rep[k] = std::min(rep[k], p[k]);
  }
  for (long r = 0; r < nrow; ++r) out.labels[r] = ulabel[row_u[r]];
  return out;
}

}  // namespace mlvs
