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
#include <climits>
#include <cstdint>
#include <cstring>
#include <thread>
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

// f(begin, end) over [0, n) split across the host's cores, one thread per 2 MB of `work` (a
// byte count) at most, so that starting threads never costs more than the pass they share
template <class F>
inline void host_parallel(long n, double work, F f) {
  const unsigned hc = std::thread::hardware_concurrency();
  const long nt = std::min<long>({(long)(hc ? hc : 1), 32L, n, (long)(work / 2e6)});
  if (nt <= 1) {
    f(0L, n);
    return;
  }
  std::vector<std::thread> th;
  const long chunk = (n + nt - 1) / nt;
  for (long t = 0; t < nt; ++t) {
    const long b = t * chunk, e = std::min(n, b + chunk);
    if (b < e) th.emplace_back(f, b, e);
  }
  for (auto& x : th) x.join();
}

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
  // row hashes: a sum of independently mixed words (no serial chain, so the loop pipelines)
  std::vector<uint64_t> hashes(nrow);
  host_parallel(nrow, (double)nrow * nb, [&](long r0, long r1) {
    for (long r = r0; r < r1; ++r) {
      const uint8_t* p = kappa + (size_t)r * nb;
      uint64_t hsh = 0;
      int k = 0;
      for (; k + 8 <= nb; k += 8) {
        uint64_t w;
        std::memcpy(&w, p + k, 8);
        const uint64_t z = (w ^ (0x9e3779b97f4a7c15ull * (uint64_t)(k + 1))) * 0xbf58476d1ce4e5b9ull;
        hsh += z ^ (z >> 32);
      }
      for (; k < nb; ++k) hsh = hsh * 31u + p[k];
      hashes[r] = hsh;
    }
  });
  for (long r = 0; r < nrow; ++r) {
    const uint8_t* p = kappa + (size_t)r * nb;
    const uint64_t hsh = hashes[r];
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
  // In that order, a mask joins the nearest centre created before it, or seeds a new one.
  // When a centre is created its distance to every later mask is evaluated (in parallel), and
  // each mask keeps the nearest centre so far (the lowest index on equal distances), so a mask
  // meets exactly the centres created before it, compared in creation order.
  std::vector<int> centre;                 // distinct-mask index of every centre
  std::vector<int> ulabel(nu, 0);
  std::vector<long> bestd(nu, LONG_MAX);   // L1 distance to the nearest centre so far
  std::vector<int> bestc(nu, -1);
  const double denom = 3.0 * nb;
  for (int pos = 0; pos < nu; ++pos) {
    const int u = order[pos];
    if (!centre.empty() && (double)bestd[u] / denom <= tau) {
      ulabel[u] = bestc[u];
      continue;
    }
    const int c = (int)centre.size();
    centre.push_back(u);
    ulabel[u] = c;
    host_parallel(nu - pos - 1, (double)(nu - pos - 1) * nb, [&](long k0, long k1) {
      for (long k = pos + 1 + k0; k < pos + 1 + k1; ++k) {
        const int v = order[k];
        const long d = l1_bytes(uptr[v], uptr[u], nb);
        if (bestc[v] < 0 || d < bestd[v]) {
          bestd[v] = d;
          bestc[v] = c;
        }
      }
    });
  }
  out.reps.assign(centre.size(), std::vector<uint8_t>(nb, 255));
  // blockwise minima over the members, the blocks split across the cores (16-byte aligned
  // ranges)
  const long nseg = (nb + 1023) / 1024;
  host_parallel(nseg, (double)nu * nb, [&](long s0, long s1) {
    const int k0 = (int)(s0 * 1024), k1 = (int)std::min<long>(nb, s1 * 1024);
    for (int u = 0; u < nu; ++u) min_bytes(out.reps[ulabel[u]].data() + k0, uptr[u] + k0, k1 - k0);
  });
  for (long r = 0; r < nrow; ++r) out.labels[r] = ulabel[row_u[r]];
  return out;
}

}  // namespace mlvs
