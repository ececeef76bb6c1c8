// partition.cpp -- element partition along a space-filling curve and the
// per-rank local meshes with their halo faces (host code, no GPU needed).
//
// The paper divides the domain into non-overlapping subdomains along a
// space-filling curve, one per process and GPU (Sec. 2.1).  Here the curve is
// the Morton (Z-order) curve of the element centroids.  A rank's local mesh
// keeps its own elements; a face whose neighbour lives on another rank becomes
// a halo face, whose remote trace arrives in the context's halo buffers.
#include <algorithm>
#include <cstdint>
#include <cstring>
#include <vector>

#include "../../include/dg.h"
#include "geometry.h"

namespace {

// spread the low 21 bits of x to every third bit
uint64_t spread3(uint64_t x) {
  uint64_t r = 0;
  for (int b = 0; b < 21; ++b) r |= ((x >> b) & 1ull) << (3 * b);
  return r;
}

struct HaloRec {
  int peer;
  long long key;  // global master element * 6 + master local face
  int elem, face, master;
};

}  // namespace

extern "C" int dg_partition_sfc(int N, int K, const double* X, int nranks, int* part) {
  if (N < 1 || K < 1 || !X || !part || nranks < 1 || nranks > K) return DG_ERR_ARG;
  const int n = N + 1, n3 = n * n * n;
  const size_t S = (size_t)K * n3;
  std::vector<double> c(3 * (size_t)K, 0.0);
  double lo[3] = {1e300, 1e300, 1e300}, hi[3] = {-1e300, -1e300, -1e300};
  for (int d = 0; d < 3; ++d)
    for (int e = 0; e < K; ++e) {
      double s = 0.0;
      for (int p = 0; p < n3; ++p) s += X[d * S + (size_t)e * n3 + p];
      s /= n3;
      c[3 * (size_t)e + d] = s;
      lo[d] = std::min(lo[d], s);
      hi[d] = std::max(hi[d], s);
    }
  std::vector<std::pair<uint64_t, int>> keys(K);
  const double cells = (double)((1u << 21) - 1);
  for (int e = 0; e < K; ++e) {
    uint64_t k = 0;
    for (int d = 0; d < 3; ++d) {
      const double span = hi[d] - lo[d];
      const double t = span > 0.0 ? (c[3 * (size_t)e + d] - lo[d]) / span : 0.0;
      const uint64_t q = (uint64_t)std::min(cells, std::max(0.0, t * cells + 0.5));
      k |= spread3(q) << d;
    }
    keys[e] = {k, e};
  }
  std::sort(keys.begin(), keys.end());
  // rank r owns the sorted positions [floor(r K / P), floor((r + 1) K / P))
  for (int r = 0; r < nranks; ++r) {
    const long long b0 = (long long)r * K / nranks, b1 = (long long)(r + 1) * K / nranks;
    for (long long i = b0; i < b1; ++i) part[keys[i].second] = r;
  }
  return DG_OK;
}

extern "C" int dg_partition_local(int K, const int* nbr, const int* nbr_face, const int* orient, const int* part,
                                  int rank, int* K_local, int* l2g, int* nbr_local, int* nbr_face_local,
                                  int* orient_local, int* n_halo, int* halo) {
  if (K < 1 || !nbr || !part || !K_local || !n_halo) return DG_ERR_ARG;
  auto nface_of = [&](int e, int l) { return nbr_face ? nbr_face[e * 6 + l] : (l ^ 1); };
  auto orient_of = [&](int e, int l) { return orient ? orient[e * 6 + l] : 0; };
  std::vector<int> g2l(K, -1);
  int Kr = 0;
  for (int e = 0; e < K; ++e)
    if (part[e] == rank) g2l[e] = Kr++;
  *K_local = Kr;
  std::vector<HaloRec> recs;
  for (int e = 0; e < K; ++e) {
    if (part[e] != rank) continue;
    for (int l = 0; l < 6; ++l) {
      const int nb = nbr[e * 6 + l];
      if (nb < 0 || part[nb] == rank) continue;
      if (nb >= K) return DG_ERR_ARG;
      // the face's master by the rule of the host geometry (global ids)
      const int l2 = nface_of(e, l);
      if (l2 < 0 || l2 > 5) return DG_ERR_ARG;
      const bool master = dg::face_is_master(e, l, nb, l2);
      const int me = master ? e : nb, ml = master ? l : l2;
      recs.push_back({part[nb], (long long)me * 6 + ml, e, l, master ? 1 : 0});
    }
  }
  // both ranks of a pair list their shared faces in the same order
  std::sort(recs.begin(), recs.end(), [](const HaloRec& a, const HaloRec& b) {
    return a.peer != b.peer ? a.peer < b.peer : a.key < b.key;
  });
  *n_halo = (int)recs.size();
  if (l2g) {
    for (int e = 0; e < K; ++e)
      if (g2l[e] >= 0) l2g[g2l[e]] = e;
  }
  if (nbr_local) {
    for (int e = 0; e < K; ++e) {
      if (g2l[e] < 0) continue;
      for (int l = 0; l < 6; ++l) {
        const int nb = nbr[e * 6 + l];
        nbr_local[g2l[e] * 6 + l] = nb < 0 ? nb : (part[nb] == rank ? g2l[nb] : 0);
      }
    }
    for (size_t h = 0; h < recs.size(); ++h)
      nbr_local[g2l[recs[h].elem] * 6 + recs[h].face] = DG_BC_HALO_BASE - (int)h;
  }
  // neighbour faces and orientations of the local elements; a halo face's
  // code carries 8 when the local element is the face's master
  if (nbr_face_local || orient_local) {
    for (int e = 0; e < K; ++e) {
      if (g2l[e] < 0) continue;
      for (int l = 0; l < 6; ++l) {
        if (nbr_face_local) nbr_face_local[g2l[e] * 6 + l] = nface_of(e, l);
        if (orient_local) orient_local[g2l[e] * 6 + l] = orient_of(e, l);
      }
    }
    if (orient_local)
      for (size_t h = 0; h < recs.size(); ++h)
        if (recs[h].master) orient_local[g2l[recs[h].elem] * 6 + recs[h].face] |= 8;
  }
  if (halo) {
    for (size_t h = 0; h < recs.size(); ++h) {
      halo[4 * h + 0] = recs[h].peer;
      halo[4 * h + 1] = g2l[recs[h].elem];
      halo[4 * h + 2] = recs[h].face;
      halo[4 * h + 3] = recs[h].master;
    }
  }
  return DG_OK;
}
