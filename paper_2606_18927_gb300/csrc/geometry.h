// geometry.h -- host-side mesh preprocessing of the GB300 DGSEM library.
//
// Builds, from node coordinates at the Legendre-Gauss-Lobatto nodes (paper
// Sec. 2.2: tensor-product LGL nodes of degree N), everything the kernels
// read: the curl-form metric terms Ja^i (Kopriva's conservative form, which
// keeps free-stream preservation on curvilinear elements), the Jacobian J,
// the face list with master-side unit normals and surface elements, and the
// wall-model sampling data (Sec. 3.1: the wall model samples the LES solution
// at the distance h_wm from the wall).
#pragma once
#include <string>
#include <vector>

namespace dg {

struct Basis {
  int N = 0, n = 0;
  std::vector<double> x, w;  // LGL nodes and weights
  std::vector<double> D;     // D[i*n + j] = l_j'(x_i)
};

// LGL nodes by the Lobatto fixed-point/Newton iteration
// x <- x - (x P_N - P_{N-1}) / ((N+1) P_N), weights 2/(N(N+1) P_N^2),
// derivative matrix in closed form.
Basis make_basis(int N);

// Lagrange basis l_j(s) (barycentric form) on the basis nodes.
void lagrange_at(const Basis& b, double s, double* l);

// neighbour codes of boundary faces (dg.h: DG_BC_WALL, DG_BC_INFLOW, DG_BC_OUTFLOW)
constexpr int BC_CODE_WALL = -1, BC_CODE_INFLOW = -2, BC_CODE_OUTFLOW = -3, BC_CODE_MIN = -3;
// halo face h of a partitioned mesh: neighbour code HALO_BASE - h (dg.h: DG_BC_HALO_BASE)
constexpr int HALO_BASE = -16;

// Orientation codes of conforming faces (dg.h): node (a, b) of one side's
// face coincides with node (a', b') of the other side's face, where
//   (s, t) = (o & 1) ? (b, a) : (a, b);  a' = (o & 2) ? N - s : s;  b' = (o & 4) ? N - t : t.
inline void orient_map(int o, int N, int a, int b, int* a2, int* b2) {
  const int s = (o & 1) ? b : a, t = (o & 1) ? a : b;
  *a2 = (o & 2) ? N - s : s;
  *b2 = (o & 4) ? N - t : t;
}
inline int orient_inverse(int o) {
  return (o & 1) ? (1 | (((o >> 2) & 1) << 1) | (((o >> 1) & 1) << 2)) : o;
}

struct Face {
  int eM, lM;  // master element and its local face
  int eS, lS;  // slave element and local face; boundary faces: eS = the code, lS = -1;
               // halo faces: eS = the halo index, lS = 1 if the local element is the master
  int o;       // interior faces: orientation from the master's face nodes to the slave's;
               // halo faces: from the local element's face nodes to the master's
};

struct Geometry {
  int N = 0, n = 0, n2 = 0, n3 = 0, K = 0;
  Basis basis;
  std::vector<int> nbr;          // [K*6]
  std::vector<int> nface;        // [K*6] the neighbour's local face (interior faces)
  std::vector<int> orient;       // [K*6] orientation code towards the neighbour's face nodes
  std::vector<double> X;         // [3][K*n3]
  std::vector<double> Ja;        // [K*n3][3 dir][3 comp]
  std::vector<double> J;         // [K*n3]
  std::vector<Face> faces;       // interior, wall, inflow / outflow, then halo faces
  int n_interior = 0, n_wall = 0, n_bc = 0, n_halo = 0;
  std::vector<int> elem_face;    // [K*6] = 16 * face id + 2 * o + side (0 master, 1 slave), o the
                                 // orientation from this element's face nodes to the master's
  std::vector<double> fgeo;      // [4][F*n2]: unit normal (master outward) and s
  std::vector<int> ws_elem;      // [n_wall*n2] element containing the sample point
  std::vector<double> ws_ref;    // [n_wall*n2][3] its reference coordinates
  std::vector<double> ws_lag;    // [n_wall*n2][3][n] Lagrange weights
};

// Returns an empty string on success, else the reason for rejecting the mesh.
// nface, orient: [K*6] neighbour faces and orientation codes, or null for the
// structured default (face l ^ 1, code 0).
std::string build_geometry(Geometry& g, int N, int K, const double* X, const int* nbr, const int* nface,
                           const int* orient, double hwm);

// The side of an interior face that is its master (whose node order indexes
// the face and whose metrics give its normal): the side with the odd local
// face (+xi, +eta, +zeta) when the two local faces differ in parity, else the
// side with the smaller (element, face) pair.  Element ids are global ones
// on partitioned meshes.
inline bool face_is_master(long long e, int l, long long nb, int l2) {
  if ((l & 1) != (l2 & 1)) return (l & 1) != 0;
  return e * 6 + l < nb * 6 + l2;
}

inline int face_node(int n, int l, int a, int b) {
  const int N = n - 1;
  switch (l) {
    case 0: return 0 + n * (a + n * b);
    case 1: return N + n * (a + n * b);
    case 2: return a + n * (0 + n * b);
    case 3: return a + n * (N + n * b);
    case 4: return a + n * (b + n * 0);
    default: return a + n * (b + n * N);
  }
}

}  // namespace dg
