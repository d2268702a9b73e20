// Host mesh-hierarchy generator (Sec. 3.1 "Grid hierarchies").
//
// Icosahedral sphere meshes refined by edge bisection.  Conventions:
//  * base icosahedron: the 12 points (+-1, +-phi, 0), (0, +-1, +-phi),
//    (+-phi, 0, +-1) in a fixed order, normalised; faces are the vertex
//    triples at mutual distance 2, in lexicographic order, each oriented
//    counter-clockwise seen from outside;
//  * face (a, b, c) with sphere-projected edge midpoints m_ab, m_bc, m_ca has
//    children 4F+0 = (a, m_ab, m_ca), 4F+1 = (m_ab, b, m_bc),
//    4F+2 = (m_ca, m_bc, c), 4F+3 = (m_bc, m_ca, m_ab): the parent of column
//    f is f / 4, which the restriction and prolongation kernels rely on;
//  * neighbour k of a face is the face across the edge opposite vertex k.
#include <cmath>
#include <cstdint>
#include <stdexcept>
#include <unordered_map>
#include <vector>

#include "hmg_internal.h"

namespace hmg {

namespace {

struct V3 {
  double x, y, z;
};

V3 sub(V3 a, V3 b) { return {a.x - b.x, a.y - b.y, a.z - b.z}; }
double dot(V3 a, V3 b) { return a.x * b.x + a.y * b.y + a.z * b.z; }
V3 cross(V3 a, V3 b) { return {a.y * b.z - a.z * b.y, a.z * b.x - a.x * b.z, a.x * b.y - a.y * b.x}; }

struct Tri {
  int32_t v[3];
};

uint64_t edge_key(int32_t a, int32_t b) {
  uint32_t lo = (uint32_t)(a < b ? a : b), hi = (uint32_t)(a < b ? b : a);
  return ((uint64_t)hi << 32) | lo;
}

void base_icosahedron(std::vector<V3>& verts, std::vector<Tri>& faces) {
  const double phi = (1.0 + std::sqrt(5.0)) / 2.0;
  const V3 pts[12] = {{-1, phi, 0}, {1, phi, 0},  {-1, -phi, 0}, {1, -phi, 0},
                      {0, -1, phi}, {0, 1, phi},  {0, -1, -phi}, {0, 1, -phi},
                      {phi, 0, -1}, {phi, 0, 1},  {-phi, 0, -1}, {-phi, 0, 1}};
  auto close2 = [&](int i, int j) {
    V3 d = sub(pts[i], pts[j]);
    return std::fabs(std::sqrt(dot(d, d)) - 2.0) < 1e-9;
  };
  faces.clear();
  for (int i = 0; i < 12; ++i)
    for (int j = i + 1; j < 12; ++j)
      for (int k = j + 1; k < 12; ++k) {
        if (!(close2(i, j) && close2(j, k) && close2(i, k))) continue;
        V3 n = cross(sub(pts[j], pts[i]), sub(pts[k], pts[i]));
        V3 s = {pts[i].x + pts[j].x + pts[k].x, pts[i].y + pts[j].y + pts[k].y,
                pts[i].z + pts[j].z + pts[k].z};
        if (dot(n, s) > 0) faces.push_back({{i, j, k}});
        else faces.push_back({{i, k, j}});
      }
  if (faces.size() != 20) throw std::runtime_error("icosahedron construction failed");
  verts.resize(12);
  for (int i = 0; i < 12; ++i) {
    double inv = 1.0 / std::sqrt(dot(pts[i], pts[i]));
    verts[i] = {pts[i].x * inv, pts[i].y * inv, pts[i].z * inv};
  }
}

void refine_once(std::vector<V3>& verts, std::vector<Tri>& faces) {
  std::unordered_map<uint64_t, int32_t> mid;
  mid.reserve(faces.size() * 2);
  auto midpoint = [&](int32_t a, int32_t b) -> int32_t {
    uint64_t key = edge_key(a, b);
    auto it = mid.find(key);
    if (it != mid.end()) return it->second;
    V3 m = {verts[a].x + verts[b].x, verts[a].y + verts[b].y, verts[a].z + verts[b].z};
    double inv = 1.0 / std::sqrt(dot(m, m));
    verts.push_back({m.x * inv, m.y * inv, m.z * inv});
    int32_t id = (int32_t)verts.size() - 1;
    mid.emplace(key, id);
    return id;
  };
  std::vector<Tri> out;
  out.reserve(faces.size() * 4);
  for (const Tri& t : faces) {
    int32_t a = t.v[0], b = t.v[1], c = t.v[2];
    int32_t mab = midpoint(a, b), mbc = midpoint(b, c), mca = midpoint(c, a);
    out.push_back({{a, mab, mca}});
    out.push_back({{mab, b, mbc}});
    out.push_back({{mca, mbc, c}});
    out.push_back({{mbc, mca, mab}});
  }
  faces.swap(out);
}

std::vector<int32_t> face_neighbours(const std::vector<Tri>& faces) {
  // edge -> first face seen; the second face completes the pair.
  std::unordered_map<uint64_t, int32_t> first;
  first.reserve(faces.size() * 2);
  std::vector<int32_t> nbr(faces.size() * 3, -1);
  for (int32_t f = 0; f < (int32_t)faces.size(); ++f) {
    for (int k = 0; k < 3; ++k) {
      uint64_t key = edge_key(faces[f].v[(k + 1) % 3], faces[f].v[(k + 2) % 3]);
      auto it = first.find(key);
      if (it == first.end()) {
        first.emplace(key, f * 3 + k);
      } else {
        int32_t g = it->second / 3, kg = it->second % 3;
        nbr[f * 3 + k] = g;
        nbr[g * 3 + kg] = f;
      }
    }
  }
  for (int32_t n : nbr)
    if (n < 0) throw std::runtime_error("mesh is not closed");
  return nbr;
}

}  // namespace

std::vector<HostLevel> build_mesh_hierarchy(int refinement, int nlevels) {
  std::vector<V3> verts;
  std::vector<Tri> faces;
  base_icosahedron(verts, faces);
  std::vector<HostLevel> by_refinement(refinement + 1);
  for (int r = 0; r <= refinement; ++r) {
    if (r > 0) refine_once(verts, faces);
    if (r < refinement + 1 - nlevels) continue;  // not part of the hierarchy
    HostLevel& L = by_refinement[r];
    L.refinement = r;
    L.ncols = (int)faces.size();
    L.verts.resize((size_t)L.ncols * 9);
    L.centroid.resize((size_t)L.ncols * 3);
    for (int f = 0; f < L.ncols; ++f) {
      double cx = 0, cy = 0, cz = 0;
      for (int k = 0; k < 3; ++k) {
        const V3& p = verts[faces[f].v[k]];
        L.verts[(size_t)f * 9 + 3 * k + 0] = p.x;
        L.verts[(size_t)f * 9 + 3 * k + 1] = p.y;
        L.verts[(size_t)f * 9 + 3 * k + 2] = p.z;
        cx += p.x;
        cy += p.y;
        cz += p.z;
      }
      L.centroid[(size_t)f * 3 + 0] = cx / 3.0;
      L.centroid[(size_t)f * 3 + 1] = cy / 3.0;
      L.centroid[(size_t)f * 3 + 2] = cz / 3.0;
    }
    L.nbr = face_neighbours(faces);
  }
  std::vector<HostLevel> levels;
  for (int lev = 0; lev < nlevels; ++lev) levels.push_back(std::move(by_refinement[refinement - lev]));
  return levels;
}

}  // namespace hmg
