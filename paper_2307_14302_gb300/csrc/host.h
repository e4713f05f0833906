// host.h -- host-side data of libdgswe: preprocessed meshes and scenarios.
#pragma once
#include <cstdint>
#include <string>
#include <vector>

#include "dgswe.h"
#include "layout.h"

namespace dg {

// A triangulation after preprocessing: counter-clockwise triangles renumbered along a Hilbert
// curve of their centroids (L2 locality of neighbour gathers), nodes renumbered by first use.
struct HostMesh {
  int nn = 0, ne = 0;
  std::vector<double> x, y;        // node coordinates, new order
  std::vector<int32_t> tri;        // [ne][3] new node indices, counter-clockwise
  std::vector<int32_t> eorig;      // new element -> caller element
  std::vector<int32_t> norig;      // new node -> caller node
  std::vector<int32_t> code;       // [ne][3]: (neighbour << 2 | its local edge), -1 land, -2-seg ocean
  std::vector<double> lnx, lny;    // [ne][3] outward normal scaled by the edge length
  std::vector<double> area;        // [ne]
  int nseg = 0;                    // 1 + largest tidal segment index used
  int nriv = 0;                    // 1 + largest river segment index used
};

int build_mesh(int nn, const double* xy, int ne, const int32_t* tri, int nb, const int32_t* bedge,
               const int32_t* btype, const int32_t* bseg, HostMesh& M, std::string& err);

void build_tables(int p, RefTab<double>& t);
void tables_to_float(const RefTab<double>& d, RefTab<float>& f);
void dubiner_eval(int p, double r, double s, double* phi, double* dphr, double* dphs);
void set_last_error(const std::string& msg);

}  // namespace dg
