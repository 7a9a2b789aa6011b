// Element partitions of a mesh for partitioned runs: recursive coordinate bisection, the
// one-element halo of a partition, and the partition's submesh (owned elements, then the halo).
#pragma once
#include <cstdint>
#include <string>
#include <vector>

#include "../../include/pcexp.h"

namespace pcexp {

// part[e] in [0, n_parts): recursive coordinate bisection of the element centroids.  A set of
// elements going to n parts is split at its floor(n/2) / n quantile along the axis of largest
// centroid extent (ties by element index), and each side recurses with its share of the parts.
void rcb_partition(const pcexp_mesh& m, int n_parts, int32_t* part);

// The elements partition k computes with: its own (ascending global index), then its halo, the
// elements of other partitions that share a face with an own element (ascending).
struct Halo {
  std::vector<int64_t> elems;
  int64_t n_owned = 0;
};
// nbr[e (dim+1) + f]: the element across local face f of e (faces matched on periodic master
// vertices, as the face list does), or -1 on a boundary face.
int face_neighbours(const pcexp_mesh& m, std::vector<int64_t>& nbr, std::string& msg);
void build_halo(const pcexp_mesh& m, const std::vector<int64_t>& nbr, const int32_t* part, int k, Halo& h);

// Submesh of a halo's elements (in that order): the vertices they use with their periodic
// masters, the tagged boundary faces among their faces, and every other face of a halo element
// that has no partner among them, tagged PCEXP_BC_SYMMETRY (its residual rows are discarded).
struct Submesh {
  int32_t dim = 2;
  std::vector<double> coords;
  std::vector<int32_t> elem_vert, vert_master, bface_vert, bface_tag;
  bool periodic = false;
  pcexp_mesh view() const;
};
int build_submesh(const pcexp_mesh& m, const Halo& h, Submesh& s, std::string& msg);

}  // namespace pcexp
