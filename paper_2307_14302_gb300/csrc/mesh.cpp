// mesh.cpp -- preprocessing of an unstructured triangulation for the device path.
//
// 1. triangles are made counter-clockwise (second and third vertices swapped when needed);
// 2. elements are sorted along a Hilbert curve through their centroids, so that the three
//    neighbours of an element sit at nearby indices and their records are L2 hits;
// 3. nodes are renumbered by first use in that order;
// 4. edges are paired by their node pair; each local edge j (vertex j -> j+1) gets a code:
//    (neighbour << 2 | neighbour's local edge), -1 for land, -2 - segment for ocean edges,
//    -2 - MAXSEG - segment for river edges (Sec. 2.1: ocean = specified elevation, land = zero
//    normal flow, river = specified normal flow).  An interior edge listed as a river edge is an
//    internal river boundary (Sec. 2.3): the river enters the triangle to the left of the listed
//    direction, whose neighbour sees a wall there; an interior land edge is a wall on both sides;
// 5. scaled outward normals ln_j = (dy, -dx) of each local edge are computed in FP64 from node
//    differences, so the two sides of an interior edge hold exactly opposite values.
#include <algorithm>
#include <cmath>
#include <cstdio>

#include "host.h"

namespace dg {

// index of (x, y) in [0, 2^order)^2 along the Hilbert curve
static uint64_t hilbert_index(uint32_t x, uint32_t y, int order) {
  const uint32_t n = 1u << order;
  uint64_t d = 0;
  for (uint32_t s = n >> 1; s > 0; s >>= 1) {
    const uint32_t rx = (x & s) ? 1u : 0u, ry = (y & s) ? 1u : 0u;
    d += (uint64_t)s * s * ((3u * rx) ^ ry);
    if (ry == 0) {  // rotate the quadrant; only bits below s matter from here on
      if (rx == 1) {
        x = n - 1 - x;
        y = n - 1 - y;
      }
      const uint32_t t = x;
      x = y;
      y = t;
    }
  }
  return d;
}

int build_mesh(int nn, const double* xy, int ne, const int32_t* tri_in, int nb, const int32_t* bedge,
               const int32_t* btype, const int32_t* bseg, HostMesh& M, std::string& err) {
  char buf[256];
  if (nn < 3 || ne < 1 || !xy || !tri_in) { err = "set_mesh: need at least 3 nodes and 1 triangle"; return DGSWE_EINVAL; }
  if (ne >= (1 << 29)) { err = "set_mesh: more than 2^29 triangles"; return DGSWE_EINVAL; }
  if (nb < 0 || (nb > 0 && (!bedge || !btype))) { err = "set_mesh: boundary arrays missing"; return DGSWE_EINVAL; }
  std::vector<int32_t> tri(tri_in, tri_in + 3 * (size_t)ne);
  for (int e = 0; e < ne; ++e) {
    int32_t* v = &tri[3 * (size_t)e];
    for (int k = 0; k < 3; ++k)
      if (v[k] < 0 || v[k] >= nn) {
        snprintf(buf, sizeof buf, "set_mesh: triangle %d has node index %d outside [0,%d)", e, v[k], nn);
        err = buf;
        return DGSWE_EINVAL;
      }
    const double cross = (xy[2 * v[1]] - xy[2 * v[0]]) * (xy[2 * v[2] + 1] - xy[2 * v[0] + 1]) -
                         (xy[2 * v[2]] - xy[2 * v[0]]) * (xy[2 * v[1] + 1] - xy[2 * v[0] + 1]);
    if (cross == 0.0 || !std::isfinite(cross)) {
      snprintf(buf, sizeof buf, "set_mesh: triangle %d is degenerate", e);
      err = buf;
      return DGSWE_EINVAL;
    }
    if (cross < 0) std::swap(v[1], v[2]);
  }
  // Hilbert order of centroids
  double xmin = 1e300, xmax = -1e300, ymin = 1e300, ymax = -1e300;
  for (int i = 0; i < nn; ++i) {
    xmin = std::min(xmin, xy[2 * i]); xmax = std::max(xmax, xy[2 * i]);
    ymin = std::min(ymin, xy[2 * i + 1]); ymax = std::max(ymax, xy[2 * i + 1]);
  }
  const double span = std::max(xmax - xmin, ymax - ymin) * (1.0 + 1e-9) + 1e-300;
  std::vector<std::pair<uint64_t, int32_t>> key(ne);
  for (int e = 0; e < ne; ++e) {
    const int32_t* v = &tri[3 * (size_t)e];
    const double cx = (xy[2 * v[0]] + xy[2 * v[1]] + xy[2 * v[2]]) / 3.0;
    const double cy = (xy[2 * v[0] + 1] + xy[2 * v[1] + 1] + xy[2 * v[2] + 1]) / 3.0;
    const uint32_t ix = (uint32_t)std::min(65535.0, std::floor((cx - xmin) / span * 65536.0));
    const uint32_t iy = (uint32_t)std::min(65535.0, std::floor((cy - ymin) / span * 65536.0));
    key[e] = {hilbert_index(ix, iy, 16), e};
  }
  std::sort(key.begin(), key.end());
  M.ne = ne;
  M.nn = nn;
  M.eorig.resize(ne);
  for (int e = 0; e < ne; ++e) M.eorig[e] = key[e].second;
  // nodes by first use
  std::vector<int32_t> nnew(nn, -1);
  M.norig.clear();
  M.norig.reserve(nn);
  M.tri.resize(3 * (size_t)ne);
  for (int e = 0; e < ne; ++e)
    for (int k = 0; k < 3; ++k) {
      const int32_t o = tri[3 * (size_t)M.eorig[e] + k];
      if (nnew[o] < 0) { nnew[o] = (int32_t)M.norig.size(); M.norig.push_back(o); }
      M.tri[3 * (size_t)e + k] = nnew[o];
    }
  for (int i = 0; i < nn; ++i)
    if (nnew[i] < 0) { nnew[i] = (int32_t)M.norig.size(); M.norig.push_back(i); }
  M.x.resize(nn);
  M.y.resize(nn);
  for (int i = 0; i < nn; ++i) { M.x[i] = xy[2 * M.norig[i]]; M.y[i] = xy[2 * M.norig[i] + 1]; }
  // pair the half edges
  struct HE { uint64_t k; int32_t e, j; };
  std::vector<HE> he(3 * (size_t)ne);
  for (int e = 0; e < ne; ++e)
    for (int j = 0; j < 3; ++j) {
      const uint32_t a = M.tri[3 * (size_t)e + j], b = M.tri[3 * (size_t)e + (j + 1) % 3];
      he[3 * (size_t)e + j] = {((uint64_t)std::min(a, b) << 32) | std::max(a, b), e, j};
    }
  std::sort(he.begin(), he.end(), [](const HE& p, const HE& q) { return p.k < q.k || (p.k == q.k && p.e < q.e); });
  std::vector<uint64_t> bkey(nb);
  std::vector<int32_t> bid(nb);
  for (int b = 0; b < nb; ++b) {
    const int32_t a0 = bedge[2 * b], b0 = bedge[2 * b + 1];
    if (a0 < 0 || a0 >= nn || b0 < 0 || b0 >= nn) { err = "set_mesh: boundary edge node out of range"; return DGSWE_EINVAL; }
    if (btype[b] != DGSWE_BT_LAND && btype[b] != DGSWE_BT_OCEAN && btype[b] != DGSWE_BT_RIVER) {
      snprintf(buf, sizeof buf, "set_mesh: boundary edge %d has unknown type %d", b, btype[b]);
      err = buf;
      return DGSWE_EINVAL;
    }
    if (btype[b] == DGSWE_BT_OCEAN && (!bseg || bseg[b] < 0 || bseg[b] >= MAXSEG)) {
      snprintf(buf, sizeof buf, "set_mesh: ocean edge %d needs a segment in [0,%d)", b, MAXSEG);
      err = buf;
      return DGSWE_EINVAL;
    }
    if (btype[b] == DGSWE_BT_RIVER && (!bseg || bseg[b] < 0 || bseg[b] >= MAXRIV)) {
      snprintf(buf, sizeof buf, "set_mesh: river edge %d needs a segment in [0,%d)", b, MAXRIV);
      err = buf;
      return DGSWE_EINVAL;
    }
    const uint32_t a = nnew[a0], c = nnew[b0];
    bkey[b] = ((uint64_t)std::min(a, c) << 32) | std::max(a, c);
    bid[b] = b;
  }
  std::sort(bid.begin(), bid.end(), [&](int32_t p, int32_t q) { return bkey[p] < bkey[q]; });
  std::vector<uint64_t> bsorted(nb);
  for (int b = 0; b < nb; ++b) bsorted[b] = bkey[bid[b]];
  M.code.assign(3 * (size_t)ne, -1);
  M.nseg = 0;
  M.nriv = 0;
  for (size_t i = 0; i < he.size();) {
    size_t k = i + 1;
    while (k < he.size() && he[k].k == he[i].k) ++k;
    if (k - i > 2) {
      err = "set_mesh: an edge is shared by more than two triangles";
      return DGSWE_EINVAL;
    }
    if (k - i == 2) {
      const HE& p = he[i];
      const HE& q = he[i + 1];
      if (M.tri[3 * (size_t)p.e + p.j] == M.tri[3 * (size_t)q.e + q.j]) {
        err = "set_mesh: neighbouring triangles traverse their shared edge in the same direction";
        return DGSWE_EINVAL;
      }
      M.code[3 * (size_t)p.e + p.j] = (q.e << 2) | q.j;
      M.code[3 * (size_t)q.e + q.j] = (p.e << 2) | p.j;
      // an interior edge listed as a boundary: a river edge (internal river boundary) lets the
      // river enter the triangle to the left of its listed direction a -> b, whose neighbour sees
      // a wall; a land edge is a wall on both sides
      auto it = std::lower_bound(bsorted.begin(), bsorted.end(), p.k);
      if (it != bsorted.end() && *it == p.k) {
        const int32_t b = bid[it - bsorted.begin()];
        if (btype[b] == DGSWE_BT_OCEAN) {
          snprintf(buf, sizeof buf, "set_mesh: boundary edge %d is interior; only river and land edges may be", b);
          err = buf;
          return DGSWE_EINVAL;
        }
        const bool p_in = M.tri[3 * (size_t)p.e + p.j] == (int32_t)nnew[bedge[2 * b]];
        const HE& in = p_in ? p : q;
        const HE& wall = p_in ? q : p;
        if (btype[b] == DGSWE_BT_RIVER) {
          M.code[3 * (size_t)in.e + in.j] = -2 - MAXSEG - bseg[b];
          M.nriv = std::max(M.nriv, bseg[b] + 1);
        } else {
          M.code[3 * (size_t)in.e + in.j] = -1;
        }
        M.code[3 * (size_t)wall.e + wall.j] = -1;
      }
    } else {
      const HE& p = he[i];
      int32_t c = -1;
      auto it = std::lower_bound(bsorted.begin(), bsorted.end(), p.k);
      if (it != bsorted.end() && *it == p.k) {
        const int32_t b = bid[it - bsorted.begin()];
        if (btype[b] == DGSWE_BT_OCEAN) {
          c = -2 - bseg[b];
          M.nseg = std::max(M.nseg, bseg[b] + 1);
        } else if (btype[b] == DGSWE_BT_RIVER) {
          c = -2 - MAXSEG - bseg[b];
          M.nriv = std::max(M.nriv, bseg[b] + 1);
        }
      }
      M.code[3 * (size_t)p.e + p.j] = c;
    }
    i = k;
  }
  // geometry
  M.lnx.resize(3 * (size_t)ne);
  M.lny.resize(3 * (size_t)ne);
  M.area.resize(ne);
  for (int e = 0; e < ne; ++e) {
    const int32_t* v = &M.tri[3 * (size_t)e];
    for (int j = 0; j < 3; ++j) {
      const int a = v[j], b = v[(j + 1) % 3];
      M.lnx[3 * (size_t)e + j] = M.y[b] - M.y[a];
      M.lny[3 * (size_t)e + j] = -(M.x[b] - M.x[a]);
    }
    M.area[e] = 0.5 * ((M.x[v[1]] - M.x[v[0]]) * (M.y[v[2]] - M.y[v[0]]) - (M.x[v[2]] - M.x[v[0]]) * (M.y[v[1]] - M.y[v[0]]));
  }
  return DGSWE_OK;
}

}  // namespace dg
