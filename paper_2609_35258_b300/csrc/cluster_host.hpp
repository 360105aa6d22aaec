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
#include <unordered_map>
#include <vector>
#if defined(__SSE2__)
#include <emmintrin.h>
#endif

namespace mlvs {

struct Clustering {
  std::vector<int> labels;               // per row
  std::vector<std::vector<uint8_t>> reps;  // per cluster, N_b entries
  int n_distinct = 0;
};

// sum_k |a_k - b_k| over n bytes
inline long l1_bytes(const uint8_t* a, const uint8_t* b, int n) {
  long s = 0;
  int k = 0;
#if defined(__SSE2__)
  __m128i acc = _mm_setzero_si128();
  for (; k + 16 <= n; k += 16) {
    const __m128i x = _mm_loadu_si128(reinterpret_cast<const __m128i*>(a + k));
    const __m128i y = _mm_loadu_si128(reinterpret_cast<const __m128i*>(b + k));
    acc = _mm_add_epi64(acc, _mm_sad_epu8(x, y));
  }
  s = _mm_cvtsi128_si64(acc) + _mm_cvtsi128_si64(_mm_unpackhi_epi64(acc, acc));
#endif
  for (; k < n; ++k) s += std::abs((int)a[k] - (int)b[k]);
  return s;
}

// r_k = min(r_k, p_k) over n bytes
inline void min_bytes(uint8_t* r, const uint8_t* p, int n) {
  int k = 0;
#if defined(__SSE2__)
  for (; k + 16 <= n; k += 16) {
    const __m128i x = _mm_loadu_si128(reinterpret_cast<const __m128i*>(r + k));
    const __m128i y = _mm_loadu_si128(reinterpret_cast<const __m128i*>(p + k));
    _mm_storeu_si128(reinterpret_cast<__m128i*>(r + k), _mm_min_epu8(x, y));
  }
#endif
  for (; k < n; ++k) r[k] = p[k] < r[k] ? p[k] : r[k];
}

inline Clustering cluster_masks(const uint8_t* kappa, long nrow, int nb, double tau) {
  Clustering out;
  out.labels.assign(nrow, 0);
  if (nrow == 0) return out;
  // distinct masks with their counts (64-bit row hash, rows compared on a hash match)
  std::unordered_multimap<uint64_t, int> idx;
  idx.reserve((size_t)nrow * 2);
  std::vector<int> row_u(nrow);
  std::vector<const uint8_t*> uptr;
  std::vector<long> cnt;
  for (long r = 0; r < nrow; ++r) {
    const uint8_t* p = kappa + (size_t)r * nb;
    // sum of independently mixed words (no serial chain, so the loop pipelines)
    uint64_t hsh = 0;
    int k = 0;
    for (; k + 8 <= nb; k += 8) {
      uint64_t w;
      std::memcpy(&w, p + k, 8);
      const uint64_t z = (w ^ (0x9e3779b97f4a7c15ull * (uint64_t)(k + 1))) * 0xbf58476d1ce4e5b9ull;
      hsh += z ^ (z >> 32);
    }
    for (; k < nb; ++k) hsh = hsh * 31u + p[k];
    int u = -1;
    auto range = idx.equal_range(hsh);
    for (auto it = range.first; it != range.second; ++it)
      if (std::memcmp(uptr[it->second], p, nb) == 0) { u = it->second; break; }
    if (u < 0) {
      u = (int)uptr.size();
      idx.emplace(hsh, u);
      uptr.push_back(p);
      cnt.push_back(0);
    }
    ++cnt[u];
    row_u[r] = u;
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
      const double d = (double)l1_bytes(uptr[u], uptr[centre[c]], nb) / denom;
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
  for (int u = 0; u < nu; ++u) min_bytes(out.reps[ulabel[u]].data(), uptr[u], nb);
  for (long r = 0; r < nrow; ++r) out.labels[r] = ulabel[row_u[r]];
  return out;
}

}  // namespace mlvs
