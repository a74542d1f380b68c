// Host-side setup of the DD solver: partition, globs, constraints, local dense
// factorizations and coarse levels (built once per matrix, Sect. 3).
#pragma once
#include <stdint.h>

#include <vector>

#include "../../include/dd_solver.h"

namespace dd {

// One subdomain of a BDDC level after setup. Local dofs are split into interior
// (I) and interface (G) dofs; the constrained Neumann problem (eq. 9) with
// a right-hand side on G only is represented by N (its G-block of the inverse),
// the coarse basis restricted to G (Phi) and the local coarse matrix KC.
struct DenseSub {
  int nI = 0, nG = 0, nc = 0;
  std::vector<double> KIIinv;  // nI x nI
  std::vector<double> E;       // nI x nG, K_II^{-1} K_IG (coarse levels only)
  std::vector<double> N;       // nG x nG
  std::vector<double> Phi;     // nG x nc (row-major)
  std::vector<double> KC;      // nc x nc
  std::vector<double> D;       // nG interface weights
  std::vector<int> cmap;       // nc global coarse dof ids
};

// A BDDC level on its own global dofs.
struct Level {
  int S = 0;                          // subdomains
  int64_t n_gamma = 0;                // interface dofs
  int n_coarse = 0;                   // coarse dofs of this level
  std::vector<int64_t> goff;          // [S+1] offsets of local interface vectors
  std::vector<int> gmap;              // flat local G -> global interface index
  std::vector<int64_t> ioff;          // [S+1] offsets of local interior vectors
  std::vector<int> gptr, gidx;        // interface CSR: copies of global dof g (flat local G positions)
  std::vector<int64_t> coff;          // [S+1] offsets of local coarse vectors
  std::vector<int> cptr, cidx;        // coarse CSR: copies of coarse dof c (flat local coarse positions)
  std::vector<DenseSub> sub;
  int n_adaptive = 0;
};

struct Mesh1 {
  int nx, ny, nz, sx, sy, sz, Sx, Sy, Sz, S;
  int fx0, fx1, fy0, fy1, fz0, fz1;   // free node box (half-open)
  int NLx, NLy, NLz, NL;              // local node grid of a subdomain
  int64_t n_free;
  std::vector<double> xc, yc, zc;
  std::vector<double> ecx, ecy, ecz;  // per element k*hy*hz/(36 hx), ... (x fastest)
  std::vector<int16_t> lidx;          // [S][NL]: >=0 interior idx, <0: -1-interface idx, INT16_MIN absent
  std::vector<int64_t> gamma_free;    // global interface index -> free node index
};

// Fast diagonalization of K_II for a constant-coefficient subdomain on a tensor mesh:
// interior nodes = P_x x P_y x P_z, K_II = k (Kz(x)My(x)Mx + Mz(x)Ky(x)Mx + Mz(x)My(x)Kx),
// K_a V_a = M_a V_a L_a with V_a^T M_a V_a = I, so K_II^{-1} = V D^{-1} V^T with
// V = Vz(x)Vy(x)Vx and D = k (Lz + Ly + Lx).
struct FdmSub {
  int n[3] = {0, 0, 0};             // |P_x|, |P_y|, |P_z|
  std::vector<double> V[3];         // n_a x n_a, row-major (V[a][i * n_a + j] = (V_a)_{ij})
  std::vector<double> Dinv;         // n_z * n_y * n_x, x fastest
};

struct HostSetup {
  Mesh1 mesh;
  Level l1;
  int local_solver = DD_LOCAL_DENSE;  // representation of K_II^{-1} on the device
  std::vector<FdmSub> fdm;             // per level-1 subdomain (local_solver == DD_LOCAL_FDM)
  // two-level coarse solve
  std::vector<double> KCinv;          // n_coarse^2 (levels == 2)
  // three-level
  int levels = 2;
  Level l2;                           // level-2 BDDC on the coarse problem
  std::vector<int> gam2_c;            // level-2 interface index -> level-1 coarse dof
  std::vector<int> imap2;             // flat level-2 interior -> level-1 coarse dof
  std::vector<double> KC3inv;         // n_coarse3^2
  // no Dirichlet face: K is semidefinite with the constants as null space (Sect. 2); the
  // coarse inverses are those of the grounded coarse matrices (first coarse dof)
  bool neumann = false;
  double setup_seconds = 0;
};

void build_host_setup(const dd_mesh_desc& md, const dd_options& opt, HostSetup& out);

}  // namespace dd
