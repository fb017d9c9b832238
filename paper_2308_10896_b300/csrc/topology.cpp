// Mesh topology, built once per topology on the host: triangle edge adjacency
// (for the silhouette test of the antialiasing) and vertex -> face lists (for
// the area-weighted vertex normals).
#include <algorithm>
#include <cstdint>
#include <vector>

namespace dsm {

// adj[3 t + e]: triangle across edge e of t (e = 0: v0v1, 1: v1v2, 2: v2v0);
// -1 boundary edge, -2 edge shared by more than two triangles.
void build_adjacency(const int32_t* tris, int T, std::vector<int32_t>& adj) {
  struct Rec { uint64_t key; int32_t slot; };
  std::vector<Rec> recs(3 * (size_t)T);
  for (int t = 0; t < T; ++t) {
    for (int e = 0; e < 3; ++e) {
      uint32_t a = (uint32_t)tris[3 * t + e], b = (uint32_t)tris[3 * t + (e == 2 ? 0 : e + 1)];
      if (a > b) std::swap(a, b);
      recs[3 * (size_t)t + e] = {((uint64_t)a << 32) | b, 3 * t + e};
    }
  }
  std::sort(recs.begin(), recs.end(), [](const Rec& x, const Rec& y) {
    return x.key < y.key || (x.key == y.key && x.slot < y.slot);
  });
  adj.assign(3 * (size_t)T, -1);
  size_t i = 0;
  while (i < recs.size()) {
    size_t j = i + 1;
    while (j < recs.size() && recs[j].key == recs[i].key) ++j;
    const size_t n = j - i;
    if (n == 2) {
      adj[recs[i].slot] = recs[i + 1].slot / 3;
      adj[recs[i + 1].slot] = recs[i].slot / 3;
    } else if (n > 2) {
      for (size_t k = i; k < j; ++k) adj[recs[k].slot] = -2;
    }
    i = j;
  }
}

// CSR lists of the faces incident to each vertex (a face appears once per
// distinct corner).
void build_vertex_faces(const int32_t* tris, int T, int V, std::vector<int32_t>& off, std::vector<int32_t>& lst) {
  off.assign((size_t)V + 1, 0);
  for (int t = 0; t < T; ++t)
    for (int k = 0; k < 3; ++k) {
      const int v = tris[3 * t + k];
      if (k > 0 && v == tris[3 * t]) continue;
      if (k > 1 && v == tris[3 * t + 1]) continue;
      off[(size_t)v + 1]++;
    }
  for (int v = 0; v < V; ++v) off[(size_t)v + 1] += off[v];
  lst.assign((size_t)off[V], 0);
  std::vector<int32_t> cur(off.begin(), off.end() - 1);
  for (int t = 0; t < T; ++t)
    for (int k = 0; k < 3; ++k) {
      const int v = tris[3 * t + k];
      if (k > 0 && v == tris[3 * t]) continue;
      if (k > 1 && v == tris[3 * t + 1]) continue;
      lst[(size_t)cur[v]++] = t;
    }
}

}  // namespace dsm
