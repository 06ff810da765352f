// Host-side construction of the icosahedral geodesic Voronoi grid and of the
// per-cell operator tables read by the CUDA stencils.
#pragma once
#include <cstdint>
#include <vector>

namespace swe {

constexpr int kSlots = 6;  // neighbour slots per cell (pentagons pad slot 5)

// Tables in the grid's final cell order.  Slot arrays are slot-major
// ([k][ncells]) so that consecutive threads (cells) read consecutive words.
struct HostGrid {
  int level = 0;
  int ng = 0;                       // number of cells N_g
  double radius = 0.0;
  std::vector<double> xyz;          // [3][ng] unit cell centres n_i
  std::vector<double> area;         // [ng] A_i [m^2]
  std::vector<int32_t> nbr;         // [6][ng] neighbour cell, pad = own index
  std::vector<double> wl;           // [6][ng] l_e/(d_e A_i)          (Laplacian)
  std::vector<double> wld;          // [ng]    -sum_k wl
  std::vector<double> nc;           // [3][6][ng] edge-value weights x l_e nu_e / A_i
  std::vector<double> ndd;          // [3][ng]    self weight of the same (D diagonal)
  std::vector<double> sdg;          // [3][ng]    S_i = sum_e l_e nu_e / A_i
  std::vector<double> vc;           // [3][6][ng] edge-value weights x l_e t_e / A_i
  std::vector<double> vd;           // [3][ng]    self weight of the same
  int64_t nA = 0;                   // structural nonzeros of J
  std::vector<int32_t> gen;         // [ng] generation index of each cell (the
                                    // order nodes are created by refinement)
  // transposed slot tables: cell j, slot k (neighbour i = nbr[k][j]) holds
  // row i's coefficient for column j (diagonals are unchanged by transposition)
  std::vector<double> wlT;          // [6][ng]
  std::vector<double> ncT;          // [3][6][ng]
  std::vector<double> vcT;          // [3][6][ng]
};

// Returns 0 on success; `err` receives a message otherwise.
int build_host_grid(int level, double radius, bool reorder, HostGrid& g, const char** err);

}  // namespace swe
