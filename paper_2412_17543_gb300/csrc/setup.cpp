// Host-side setup (Sect. 3): partition of a tensor-product Q1 mesh into blocks,
// interior/interface split, globs and coarse dofs, dense local factorizations,
// coarse levels. Runs once per matrix; everything per subdomain is independent
// and parallelised with OpenMP.
#include "setup.h"

#include <omp.h>

#include <algorithm>
#include <chrono>
#include <climits>
#include <cmath>
#include <map>
#include <string>

#include "common.h"
#include "hostla.h"
#include "lobpcg.h"

namespace dd {

namespace {

enum { GLOB_FACE = 0, GLOB_EDGE = 1, GLOB_CORNER = 2 };

int glob_kind(int mult) { return mult <= 2 ? GLOB_FACE : (mult < 8 ? GLOB_EDGE : GLOB_CORNER); }

struct Globs {
  std::vector<std::vector<int>> subs;     // sharing set (sorted subdomain ids)
  std::vector<std::vector<int64_t>> dofs; // global interface dofs (ascending)
  std::vector<int> kind;
};

// Globs = interface dofs grouped by their sharing set, ordered by first dof (Sect. 3.2).
template <class F>
Globs make_globs(int64_t n_gamma, F sharing) {
  Globs gl;
  std::map<std::vector<int>, int> id;
  std::vector<int> s;
  for (int64_t g = 0; g < n_gamma; ++g) {
    s.clear();
    sharing(g, s);
    auto it = id.find(s);
    int k;
    if (it == id.end()) {
      k = (int)gl.subs.size();
      id.emplace(s, k);
      gl.subs.push_back(s);
      gl.dofs.emplace_back();
      gl.kind.push_back(glob_kind((int)s.size()));
    } else {
      k = it->second;
    }
    gl.dofs[k].push_back(g);
  }
  return gl;
}

struct CoarseDof {
  int glob;
  std::vector<double> row;  // over the glob's dofs
};

// Constraint rows of subdomain s (nc_s x nG_s) from the coarse dofs touching it.
void subdomain_constraints(const Level& L, int s, const Globs& gl, const std::vector<CoarseDof>& cd,
                           const std::vector<std::vector<int>>& cdofs_of_sub, std::vector<double>& C) {
  int nG = (int)(L.goff[s + 1] - L.goff[s]);
  const int* gm = L.gmap.data() + L.goff[s];
  const auto& mine = cdofs_of_sub[s];
  C.assign((size_t)mine.size() * nG, 0.0);
  for (size_t r = 0; r < mine.size(); ++r) {
    const CoarseDof& c = cd[mine[r]];
    const auto& dofs = gl.dofs[c.glob];
    for (size_t t = 0; t < dofs.size(); ++t) {
      int pos = (int)(std::lower_bound(gm, gm + nG, (int)dofs[t]) - gm);
      if (pos >= nG || gm[pos] != dofs[t]) throw Error(DD_INVALID_ARG, "glob dof not in subdomain interface");
      C[r * nG + pos] = c.row[t];
    }
  }
}

// Phase A of one subdomain: K_II^{-1} and the local Schur complement
// S = K_GG - K_GI K_II^{-1} K_IG (Sect. 3.1); E = K_II^{-1} K_IG on coarse levels.
bool dense_schur(int nloc, const double* K, const std::vector<int>& I, const std::vector<int>& G, bool needE,
                 DenseSub& out, std::vector<double>& S) {
  int nI = (int)I.size(), nG = (int)G.size();
  out.nI = nI;
  out.nG = nG;
  std::vector<double> KII((size_t)nI * nI), KIG((size_t)nI * nG);
  S.assign((size_t)nG * nG, 0.0);
  for (int a = 0; a < nI; ++a) {
    for (int b = 0; b < nI; ++b) KII[(size_t)a * nI + b] = K[(size_t)I[a] * nloc + I[b]];
    for (int b = 0; b < nG; ++b) KIG[(size_t)a * nG + b] = K[(size_t)I[a] * nloc + G[b]];
  }
  for (int a = 0; a < nG; ++a)
    for (int b = 0; b < nG; ++b) S[(size_t)a * nG + b] = K[(size_t)G[a] * nloc + G[b]];
  if (nI > 0) {
    if (!la::cholesky(nI, KII.data())) return false;
    std::vector<double> Linv((size_t)nI * nI);
    la::tri_inv_lower(nI, KII.data(), Linv.data());
    std::vector<double> LT((size_t)nI * nI);
    for (int a = 0; a < nI; ++a)
      for (int b = 0; b < nI; ++b) LT[(size_t)a * nI + b] = Linv[(size_t)b * nI + a];
    out.KIIinv.assign((size_t)nI * nI, 0.0);
    for (int a = 0; a < nI; ++a)
      for (int b = 0; b <= a; ++b) {
        const double* ra = LT.data() + (size_t)a * nI;
        const double* rb = LT.data() + (size_t)b * nI;
        double sacc = 0.0;
        for (int k = a; k < nI; ++k) sacc += ra[k] * rb[k];
        out.KIIinv[(size_t)a * nI + b] = sacc;
        out.KIIinv[(size_t)b * nI + a] = sacc;
      }
    std::vector<double> X((size_t)nI * nG), XT((size_t)nG * nI);
    la::trmm_lower(nI, nG, Linv.data(), KIG.data(), X.data());
    for (int a = 0; a < nI; ++a)
      for (int b = 0; b < nG; ++b) XT[(size_t)b * nI + a] = X[(size_t)a * nG + b];
    la::gemm_nt(nG, nG, nI, -1.0, XT.data(), XT.data(), 1.0, S.data());
    if (needE) {
      out.E.resize((size_t)nI * nG);
      la::gemm_nn(nI, nG, nI, LT.data(), X.data(), out.E.data());
    }
  }
  for (int a = 0; a < nG; ++a)  // symmetrize
    for (int b = 0; b < a; ++b) {
      double v = 0.5 * (S[(size_t)a * nG + b] + S[(size_t)b * nG + a]);
      S[(size_t)a * nG + b] = S[(size_t)b * nG + a] = v;
    }
  return true;
}

// Phase C of one subdomain: the constrained Neumann problem of eq. 9 with a
// right-hand side on G. With S^ = S + rho C^T C (equal to S on ker C):
// N = S^{-1} - S^{-1}C^T (C S^{-1} C^T)^{-1} C S^{-1}, Phi = S^{-1} C^T (C S^{-1} C^T)^{-1},
// KC = Phi^T S Phi = (C S^{-1} C^T)^{-1} - rho I.
bool dense_bddc(const std::vector<double>& S, const std::vector<double>& C, int nc, DenseSub& out) {
  int nG = out.nG;
  out.nc = nc;
  std::vector<double> Sh = S;
  double rho = 0.0;
  if (nc > 0) {
    double trS = 0.0, trC = 0.0;
    for (int a = 0; a < nG; ++a) trS += S[(size_t)a * nG + a];
    for (size_t t = 0; t < C.size(); ++t) trC += C[t] * C[t];
    rho = trS / std::max(trC, 1e-300);
    for (int r = 0; r < nc; ++r) {
      const double* cr = C.data() + (size_t)r * nG;
      for (int a = 0; a < nG; ++a) {
        if (cr[a] == 0.0) continue;
        double ca = rho * cr[a];
        for (int b = 0; b < nG; ++b) Sh[(size_t)a * nG + b] += ca * cr[b];
      }
    }
  }
  std::vector<double> Shinv((size_t)nG * nG);
  if (!la::spd_inverse(nG, Sh.data(), Shinv.data())) return false;
  if (nc == 0) {
    out.N = Shinv;
    return true;
  }
  std::vector<double> Xc((size_t)nG * nc), Y((size_t)nc * nc), Yinv((size_t)nc * nc);
  la::gemm_nt(nG, nc, nG, 1.0, Shinv.data(), C.data(), 0.0, Xc.data());  // S^{-1} C^T
  la::gemm_nn(nc, nc, nG, C.data(), Xc.data(), Y.data());                // C S^{-1} C^T
  for (int a = 0; a < nc; ++a)
    for (int b = 0; b < a; ++b) {
      double v = 0.5 * (Y[(size_t)a * nc + b] + Y[(size_t)b * nc + a]);
      Y[(size_t)a * nc + b] = Y[(size_t)b * nc + a] = v;
    }
  if (!la::spd_inverse(nc, Y.data(), Yinv.data())) return false;
  out.Phi.resize((size_t)nG * nc);
  la::gemm_nn(nG, nc, nc, Xc.data(), Yinv.data(), out.Phi.data());
  out.N = Shinv;
  la::gemm_nt(nG, nG, nc, -1.0, out.Phi.data(), Xc.data(), 1.0, out.N.data());
  for (int a = 0; a < nG; ++a)
    for (int b = 0; b < a; ++b) {
      double v = 0.5 * (out.N[(size_t)a * nG + b] + out.N[(size_t)b * nG + a]);
      out.N[(size_t)a * nG + b] = out.N[(size_t)b * nG + a] = v;
    }
  out.KC = Yinv;
  for (int a = 0; a < nc; ++a) out.KC[(size_t)a * nc + a] -= rho;
  for (int a = 0; a < nc; ++a)
    for (int b = 0; b < a; ++b) {
      double v = 0.5 * (out.KC[(size_t)a * nc + b] + out.KC[(size_t)b * nc + a]);
      out.KC[(size_t)a * nc + b] = out.KC[(size_t)b * nc + a] = v;
    }
  return true;
}

// CSR listing, for every global dof, the flat local positions of its copies (subdomains ascending).
void build_copy_csr(int64_t n, const std::vector<int64_t>& off, const std::vector<int>& map, std::vector<int>& ptr,
                    std::vector<int>& idx) {
  ptr.assign(n + 1, 0);
  for (size_t k = 0; k < map.size(); ++k) ptr[map[k] + 1]++;
  for (int64_t g = 0; g < n; ++g) ptr[g + 1] += ptr[g];
  idx.assign(map.size(), 0);
  std::vector<int> fill(ptr.begin(), ptr.end() - 1);
  for (size_t k = 0; k < map.size(); ++k) idx[fill[map[k]]++] = (int)k;  // k ascending => subdomains ascending
  (void)off;
}

// Select coarse dofs from globs by kind (Sect. 3.2: corners = point values, edges/faces = averages).
std::vector<CoarseDof> select_coarse(const Globs& gl, bool corners, bool edges, bool faces) {
  std::vector<CoarseDof> cd;
  for (size_t g = 0; g < gl.kind.size(); ++g) {
    int k = gl.kind[g];
    if ((k == GLOB_CORNER && corners) || (k == GLOB_EDGE && edges) || (k == GLOB_FACE && faces)) {
      size_t m = gl.dofs[g].size();
      cd.push_back({(int)g, std::vector<double>(m, 1.0 / (double)m)});
    }
  }
  return cd;
}

// Local positions (in subdomain s's interface list) of a glob's dofs.
std::vector<int> glob_positions(const Level& L, int s, const std::vector<int64_t>& dofs) {
  int nG = (int)(L.goff[s + 1] - L.goff[s]);
  const int* gm = L.gmap.data() + L.goff[s];
  std::vector<int> pos(dofs.size());
  for (size_t t = 0; t < dofs.size(); ++t) {
    int p = (int)(std::lower_bound(gm, gm + nG, (int)dofs[t]) - gm);
    if (p >= nG || gm[p] != dofs[t]) throw Error(DD_INVALID_ARG, "glob dof not in subdomain interface");
    pos[t] = p;
  }
  return pos;
}

// Schur complement of S onto the positions F (all other rows/columns eliminated).
bool face_schur(int nG, const std::vector<double>& S, const std::vector<int>& F, std::vector<double>& A) {
  int m = (int)F.size();
  std::vector<char> inF(nG, 0);
  for (int p : F) inF[p] = 1;
  std::vector<int> R;
  for (int p = 0; p < nG; ++p)
    if (!inF[p]) R.push_back(p);
  int r = (int)R.size();
  A.assign((size_t)m * m, 0.0);
  for (int a = 0; a < m; ++a)
    for (int b = 0; b < m; ++b) A[(size_t)a * m + b] = S[(size_t)F[a] * nG + F[b]];
  if (r == 0) return true;
  std::vector<double> SRR((size_t)r * r), SRF((size_t)r * m), Linv((size_t)r * r), X((size_t)r * m),
      XT((size_t)m * r);
  for (int a = 0; a < r; ++a) {
    for (int b = 0; b < r; ++b) SRR[(size_t)a * r + b] = S[(size_t)R[a] * nG + R[b]];
    for (int b = 0; b < m; ++b) SRF[(size_t)a * m + b] = S[(size_t)R[a] * nG + F[b]];
  }
  if (!la::cholesky(r, SRR.data())) return false;
  la::tri_inv_lower(r, SRR.data(), Linv.data());
  la::trmm_lower(r, m, Linv.data(), SRF.data(), X.data());
  for (int a = 0; a < r; ++a)
    for (int b = 0; b < m; ++b) XT[(size_t)b * r + a] = X[(size_t)a * m + b];
  la::gemm_nt(m, m, r, -1.0, XT.data(), XT.data(), 1.0, A.data());
  for (int a = 0; a < m; ++a)
    for (int b = 0; b < a; ++b) {
      double v = 0.5 * (A[(size_t)a * m + b] + A[(size_t)b * m + a]);
      A[(size_t)a * m + b] = A[(size_t)b * m + a] = v;
    }
  return true;
}

// Adaptive constraints of one face shared by two subdomains (Sect. 3.3, eqs. 10, 12),
// posed on their common interface (the face with the edges and corners it touches).
// As, At: Schur complements of the two subdomains onto the common interface; ws, wt: BDDC weights
// there; cq: the initial coarse dofs of the common interface (rows over its dofs). Pi projects onto
// the space where both copies agree in every initial coarse dof, E averages the copies with the
// weights. Eigenvectors with lambda > tau (largest first, at most maxr) give c = w^T Pi (I-E)^T A
// (I-E) Pi; its entries on the face (positions fpos, first copy) form a row, orthogonalized against
// the face average and the rows before it.
std::vector<std::vector<double>> face_eigen_rows(const std::vector<double>& As, const std::vector<double>& At,
                                                 const std::vector<double>& ws, const std::vector<double>& wt,
                                                 const std::vector<std::vector<double>>& cq,
                                                 const std::vector<int>& fpos, double tau, int maxr) {
  const int m = (int)ws.size(), n = 2 * m;
  std::vector<double> A((size_t)n * n, 0.0), IE((size_t)n * n, 0.0), Pi((size_t)n * n, 0.0);
  for (int a = 0; a < m; ++a)
    for (int b = 0; b < m; ++b) {
      A[(size_t)a * n + b] = As[(size_t)a * m + b];
      A[(size_t)(m + a) * n + m + b] = At[(size_t)a * m + b];
    }
  for (int a = 0; a < m; ++a) {  // I - E, E = [[Ws, Wt], [Ws, Wt]]
    IE[(size_t)a * n + a] += 1.0;
    IE[(size_t)(m + a) * n + m + a] += 1.0;
    IE[(size_t)a * n + a] -= ws[a];
    IE[(size_t)a * n + m + a] -= wt[a];
    IE[(size_t)(m + a) * n + a] -= ws[a];
    IE[(size_t)(m + a) * n + m + a] -= wt[a];
  }
  // orthonormal basis of the jumps (c, -c) of the initial coarse dofs (modified Gram-Schmidt)
  std::vector<std::vector<double>> Qo;
  for (const auto& c : cq) {
    std::vector<double> q(n);
    for (int a = 0; a < m; ++a) {
      q[a] = c[a];
      q[m + a] = -c[a];
    }
    double n0 = 0.0;
    for (double v : q) n0 += v * v;
    n0 = std::sqrt(n0);
    for (const auto& b : Qo) {
      double d = 0.0;
      for (int a = 0; a < n; ++a) d += b[a] * q[a];
      for (int a = 0; a < n; ++a) q[a] -= d * b[a];
    }
    double n1 = 0.0;
    for (double v : q) n1 += v * v;
    n1 = std::sqrt(n1);
    if (n1 <= 1e-12 * n0) continue;
    for (double& v : q) v /= n1;
    Qo.push_back(q);
  }
  for (int a = 0; a < n; ++a)
    for (int b = 0; b < n; ++b) {
      double v = (a == b ? 1.0 : 0.0);
      for (const auto& q : Qo) v -= q[a] * q[b];
      Pi[(size_t)a * n + b] = v;
    }
  std::vector<double> T1((size_t)n * n), T2((size_t)n * n), Lhs((size_t)n * n), Rhs((size_t)n * n);
  // Lhs = Pi IE^T A IE Pi ; Rhs = Pi A Pi
  std::vector<double> IEPi((size_t)n * n);
  la::gemm_nn(n, n, n, IE.data(), Pi.data(), IEPi.data());
  la::gemm_nn(n, n, n, A.data(), IEPi.data(), T1.data());           // A IE Pi
  std::vector<double> IEPiT((size_t)n * n);
  for (int a = 0; a < n; ++a)
    for (int b = 0; b < n; ++b) IEPiT[(size_t)a * n + b] = IEPi[(size_t)b * n + a];
  la::gemm_nn(n, n, n, IEPiT.data(), T1.data(), Lhs.data());
  la::gemm_nn(n, n, n, A.data(), Pi.data(), T1.data());
  la::gemm_nn(n, n, n, Pi.data(), T1.data(), Rhs.data());
  for (int a = 0; a < n; ++a)
    for (int b = 0; b < a; ++b) {
      double v = 0.5 * (Lhs[(size_t)a * n + b] + Lhs[(size_t)b * n + a]);
      Lhs[(size_t)a * n + b] = Lhs[(size_t)b * n + a] = v;
      v = 0.5 * (Rhs[(size_t)a * n + b] + Rhs[(size_t)b * n + a]);
      Rhs[(size_t)a * n + b] = Rhs[(size_t)b * n + a] = v;
    }
  // restrict to the range of Rhs (drops ker Pi and the common null space)
  std::vector<double> lam(n), U((size_t)n * n), Rw = Rhs;
  la::sym_eig(n, Rw.data(), lam.data(), U.data());
  std::vector<int> keep;
  for (int a = 0; a < n; ++a)
    if (lam[a] > 1e-12 * lam[n - 1]) keep.push_back(a);
  int r = (int)keep.size();
  std::vector<std::vector<double>> rows;
  if (r == 0) return rows;
  std::vector<double> T((size_t)n * r);
  for (int a = 0; a < n; ++a)
    for (int j = 0; j < r; ++j) T[(size_t)a * r + j] = U[(size_t)a * n + keep[j]] / std::sqrt(lam[keep[j]]);
  std::vector<double> LT((size_t)n * r), Cm((size_t)r * r);
  la::gemm_nn(n, r, n, Lhs.data(), T.data(), LT.data());
  for (int i = 0; i < r; ++i)
    for (int j = 0; j < r; ++j) {
      double sacc = 0.0;
      for (int a = 0; a < n; ++a) sacc += T[(size_t)a * r + i] * LT[(size_t)a * r + j];
      Cm[(size_t)i * r + j] = sacc;
    }
  std::vector<double> mu(r), V((size_t)r * r);
  la::sym_eig(r, Cm.data(), mu.data(), V.data());
  const int mf = (int)fpos.size();
  std::vector<std::vector<double>> basis;
  {
    std::vector<double> a0(mf, 1.0 / std::sqrt((double)mf));
    basis.push_back(a0);
  }
  for (int j = r - 1; j >= 0 && (int)rows.size() < maxr; --j) {
    if (!(mu[j] > tau)) break;
    std::vector<double> w(n, 0.0);
    for (int a = 0; a < n; ++a)
      for (int i = 0; i < r; ++i) w[a] += T[(size_t)a * r + i] * V[(size_t)i * r + j];
    std::vector<double> row(mf, 0.0);  // c = w^T Lhs on the face, first copy
    for (int b = 0; b < mf; ++b) {
      double sacc = 0.0;
      for (int a = 0; a < n; ++a) sacc += w[a] * Lhs[(size_t)a * n + fpos[b]];
      row[b] = sacc;
    }
    double n0 = 0.0;
    for (double v : row) n0 += v * v;
    n0 = std::sqrt(n0);
    if (n0 == 0.0) continue;
    for (const auto& bv : basis) {
      double d = 0.0;
      for (int b = 0; b < mf; ++b) d += bv[b] * row[b];
      for (int b = 0; b < mf; ++b) row[b] -= d * bv[b];
    }
    double n1 = 0.0;
    for (double v : row) n1 += v * v;
    n1 = std::sqrt(n1);
    if (n1 < 1e-10 * n0) continue;
    for (double& v : row) v /= n1;
    basis.push_back(row);
    rows.push_back(row);
  }
  return rows;
}

struct AdaptiveOpts {
  bool on = false;
  double tau = 10.0;
  int max_per_face = 10;
  bool lobpcg = false;  // face eigenproblems by the batched device LOBPCG (else dense, on the host)
  int lobpcg_iters = 15;
};

// Orthonormal basis (modified Gram-Schmidt, dependent columns dropped) of the jumps (c, -c)
// of the initial coarse dofs c of a common interface of m dofs: the span that Pi removes.
std::vector<std::vector<double>> jump_basis(int m, const std::vector<std::vector<double>>& cq) {
  const int n = 2 * m;
  std::vector<std::vector<double>> Qo;
  for (const auto& c : cq) {
    std::vector<double> q(n);
    for (int a = 0; a < m; ++a) {
      q[a] = c[a];
      q[m + a] = -c[a];
    }
    double n0 = 0.0;
    for (double v : q) n0 += v * v;
    n0 = std::sqrt(n0);
    for (const auto& b : Qo) {
      double d = 0.0;
      for (int a = 0; a < n; ++a) d += b[a] * q[a];
      for (int a = 0; a < n; ++a) q[a] -= d * b[a];
    }
    double n1 = 0.0;
    for (double v : q) n1 += v * v;
    n1 = std::sqrt(n1);
    if (n1 <= 1e-12 * n0) continue;
    for (double& v : q) v /= n1;
    Qo.push_back(q);
  }
  return Qo;
}

// Constraint rows of one face from eigenpairs of eq. 10 (theta descending): for theta_j > tau
// (at most maxr), c = w_j^T Lhs, i.e. (Lhs w_j) on the face dofs of the first copy (fpos),
// orthogonalized against the face average and the rows before it (dropped below 1e-10).
std::vector<std::vector<double>> rows_from_pairs(const std::vector<double>& theta, const std::vector<double>& LW,
                                                 int n, const std::vector<int>& fpos, double tau, int maxr) {
  const int mf = (int)fpos.size();
  std::vector<std::vector<double>> basis, rows;
  basis.push_back(std::vector<double>(mf, 1.0 / std::sqrt((double)mf)));
  for (size_t j = 0; j < theta.size() && (int)rows.size() < maxr; ++j) {
    if (!(theta[j] > tau)) break;
    std::vector<double> row(mf);
    for (int b = 0; b < mf; ++b) row[b] = LW[j * n + fpos[b]];
    double n0 = 0.0;
    for (double v : row) n0 += v * v;
    n0 = std::sqrt(n0);
    if (n0 == 0.0) continue;
    for (const auto& bv : basis) {
      double d = 0.0;
      for (int b = 0; b < mf; ++b) d += bv[b] * row[b];
      for (int b = 0; b < mf; ++b) row[b] -= d * bv[b];
    }
    double n1 = 0.0;
    for (double v : row) n1 += v * v;
    n1 = std::sqrt(n1);
    if (n1 < 1e-10 * n0) continue;
    for (double& v : row) v /= n1;
    basis.push_back(row);
    rows.push_back(row);
  }
  return rows;
}

// Weights, constraints and dense pipelines of a level whose subdomain matrices are given:
// phase A (Schur complements), weights, optional adaptive face constraints, phase C (BDDC).
template <class KFn, class DiagFn>
void finish_level(Level& L, const Globs& gl, std::vector<CoarseDof> cd, int weights, KFn kloc_fn, DiagFn diag_fn,
                  const std::vector<int>& nloc, const std::vector<std::vector<int>>& Iloc,
                  const std::vector<std::vector<int>>& Gloc, bool needE, const AdaptiveOpts& ad, const char* what) {
  L.sub.assign(L.S, DenseSub());
  std::vector<std::vector<double>> S(L.S);
  int failed = -1;
#pragma omp parallel for schedule(dynamic, 1)
  for (int s = 0; s < L.S; ++s) {
    std::vector<double> K;
    kloc_fn(s, K);
    if (!dense_schur(nloc[s], K.data(), Iloc[s], Gloc[s], needE, L.sub[s], S[s])) {
#pragma omp critical
      failed = s;
    }
  }
  if (failed >= 0)
    throw Error(DD_SINGULAR_LOCAL, std::string(what) + ": non-positive pivot in K_II of subdomain " +
                                       std::to_string(failed));
  // weights D_i (Sect. 3.2): card = inverse multiplicity, diag = share of the diagonal entries
  std::vector<double> dsum(L.n_gamma, 0.0);
  std::vector<std::vector<double>> diag(L.S);
  for (int s = 0; s < L.S; ++s) {
    diag_fn(s, diag[s]);
    if (weights == DD_WEIGHTS_DIAG)
      for (size_t j = 0; j < Gloc[s].size(); ++j) dsum[L.gmap[L.goff[s] + j]] += diag[s][Gloc[s][j]];
  }
  for (int s = 0; s < L.S; ++s) {
    DenseSub& ds = L.sub[s];
    ds.D.resize(Gloc[s].size());
    for (size_t j = 0; j < Gloc[s].size(); ++j) {
      int g = L.gmap[L.goff[s] + j];
      ds.D[j] = weights == DD_WEIGHTS_DIAG ? diag[s][Gloc[s][j]] / dsum[g]
                                           : 1.0 / (double)(L.gptr[g + 1] - L.gptr[g]);
    }
  }
  // adaptive face constraints (Sect. 3.3), inserted after each face's average
  if (ad.on) {
    std::vector<int> faces;
    for (size_t g = 0; g < gl.kind.size(); ++g)
      if (gl.kind[g] == GLOB_FACE && gl.subs[g].size() == 2 && gl.dofs[g].size() >= 2) faces.push_back((int)g);
    std::vector<std::vector<int>> globs_of_sub(L.S);
    for (size_t g = 0; g < gl.subs.size(); ++g)
      for (int s : gl.subs[g]) globs_of_sub[s].push_back((int)g);
    std::vector<char> initial(gl.kind.size(), 0);
    for (const CoarseDof& c : cd) initial[c.glob] = 1;
    std::vector<std::vector<std::vector<double>>> extra(faces.size());
    std::vector<FaceProblem> fprob(ad.lobpcg ? faces.size() : 0);
    std::vector<std::vector<int>> fposs(ad.lobpcg ? faces.size() : 0);
    int bad = -1;
#pragma omp parallel for schedule(dynamic, 1)
    for (int f = 0; f < (int)faces.size(); ++f) {
      int g = faces[f];
      int s = gl.subs[g][0], t = gl.subs[g][1];
      // common interface of s and t: every glob whose sharing set holds both
      std::vector<int> closure;
      for (int g2 : globs_of_sub[s])
        if (std::binary_search(gl.subs[g2].begin(), gl.subs[g2].end(), t)) closure.push_back(g2);
      std::vector<int64_t> dofs;
      for (int g2 : closure) dofs.insert(dofs.end(), gl.dofs[g2].begin(), gl.dofs[g2].end());
      std::sort(dofs.begin(), dofs.end());
      std::vector<int> Fs = glob_positions(L, s, dofs), Ft = glob_positions(L, t, dofs);
      std::vector<double> As, At;
      if (!face_schur(L.sub[s].nG, S[s], Fs, As) || !face_schur(L.sub[t].nG, S[t], Ft, At)) {
#pragma omp critical
        bad = g;
        continue;
      }
      const int m = (int)dofs.size();
      std::vector<double> ws(m), wt(m);
      for (int a = 0; a < m; ++a) {
        ws[a] = L.sub[s].D[Fs[a]];
        wt[a] = L.sub[t].D[Ft[a]];
      }
      std::vector<std::vector<double>> cq;
      for (int g2 : closure) {
        if (!initial[g2]) continue;
        std::vector<double> c(m, 0.0);
        for (int64_t d : gl.dofs[g2])
          c[std::lower_bound(dofs.begin(), dofs.end(), d) - dofs.begin()] = 1.0 / (double)gl.dofs[g2].size();
        cq.push_back(c);
      }
      std::vector<int> fpos;
      for (int64_t d : gl.dofs[g]) fpos.push_back((int)(std::lower_bound(dofs.begin(), dofs.end(), d) - dofs.begin()));
      if (!ad.lobpcg) {
        extra[f] = face_eigen_rows(As, At, ws, wt, cq, fpos, ad.tau, ad.max_per_face);
        continue;
      }
      // the pencil for the device LOBPCG: both Schur complements, weights, jump basis, and
      // whether both subdomains float (A_s 1 = A_t 1 = 0: the common constant is removed too)
      FaceProblem& P = fprob[f];
      P.m = m;
      auto annihilates_constants = [&](const std::vector<double>& M) {
        double fro = 0.0, r2 = 0.0;
        for (double v : M) fro += v * v;
        for (int a = 0; a < m; ++a) {
          double r = 0.0;
          for (int b = 0; b < m; ++b) r += M[(size_t)a * m + b];
          r2 += r * r;
        }
        return std::sqrt(r2) <= 1e-10 * std::sqrt(fro) * std::sqrt((double)m);
      };
      P.floating = annihilates_constants(As) && annihilates_constants(At) ? 1 : 0;
      auto Qo = jump_basis(m, cq);
      P.nq = (int)Qo.size();
      for (const auto& q : Qo) P.Q.insert(P.Q.end(), q.begin(), q.end());
      P.As = std::move(As);
      P.At = std::move(At);
      P.ws = std::move(ws);
      P.wt = std::move(wt);
      fposs[f] = std::move(fpos);
    }
    if (bad >= 0) throw Error(DD_SINGULAR_LOCAL, std::string(what) + ": singular face Schur complement");
    if (ad.lobpcg) {
      std::vector<FaceResult> res;
      face_lobpcg_batch(fprob, std::min(ad.max_per_face, LOBPCG_MAXK), ad.lobpcg_iters, res);
#pragma omp parallel for schedule(dynamic, 8)
      for (int f = 0; f < (int)faces.size(); ++f)
        extra[f] = rows_from_pairs(res[f].theta, res[f].LX, 2 * fprob[f].m, fposs[f], ad.tau, ad.max_per_face);
    }
    std::vector<std::vector<std::vector<double>>> by_glob(gl.kind.size());
    for (size_t f = 0; f < faces.size(); ++f) by_glob[faces[f]] = std::move(extra[f]);
    std::vector<CoarseDof> cd2;
    for (const CoarseDof& c : cd) {
      cd2.push_back(c);
      for (auto& row : by_glob[c.glob]) {
        cd2.push_back({c.glob, row});
        L.n_adaptive++;
      }
    }
    cd.swap(cd2);
  }
  L.n_coarse = (int)cd.size();
  std::vector<std::vector<int>> cdofs_of_sub(L.S);
  for (size_t c = 0; c < cd.size(); ++c)
    for (int s : gl.subs[cd[c].glob]) cdofs_of_sub[s].push_back((int)c);
#pragma omp parallel for schedule(dynamic, 1)
  for (int s = 0; s < L.S; ++s) {
    std::vector<double> C;
    subdomain_constraints(L, s, gl, cd, cdofs_of_sub, C);
    DenseSub& ds = L.sub[s];
    if (!dense_bddc(S[s], C, (int)cdofs_of_sub[s].size(), ds)) {
#pragma omp critical
      failed = s;
    }
    ds.cmap = cdofs_of_sub[s];
    std::vector<double>().swap(S[s]);
  }
  if (failed >= 0)
    throw Error(DD_SINGULAR_LOCAL, std::string(what) + ": singular constrained problem in subdomain " +
                                       std::to_string(failed));
  // coarse copy CSR
  L.coff.assign(L.S + 1, 0);
  for (int s = 0; s < L.S; ++s) L.coff[s + 1] = L.coff[s] + L.sub[s].nc;
  std::vector<int> cflat(L.coff[L.S]);
  for (int s = 0; s < L.S; ++s)
    for (int c = 0; c < L.sub[s].nc; ++c) cflat[L.coff[s] + c] = L.sub[s].cmap[c];
  build_copy_csr(L.n_coarse, L.coff, cflat, L.cptr, L.cidx);
}

std::vector<double> assemble_coarse(const Level& L) {
  size_t n = L.n_coarse;
  std::vector<double> KC(n * n, 0.0);
  for (int s = 0; s < L.S; ++s) {
    const DenseSub& d = L.sub[s];
    for (int a = 0; a < d.nc; ++a)
      for (int b = 0; b < d.nc; ++b) KC[(size_t)d.cmap[a] * n + d.cmap[b]] += d.KC[(size_t)a * d.nc + b];
  }
  return KC;
}

}  // namespace

void build_host_setup(const dd_mesh_desc& md, const dd_options& opt, HostSetup& H) {
  auto t0 = std::chrono::steady_clock::now();
  DD_REQUIRE(md.nx >= 1 && md.ny >= 1 && md.nz >= 1, "mesh sizes must be positive");
  DD_REQUIRE(md.xc && md.yc && md.zc, "coordinate arrays required");
  DD_REQUIRE(md.sub_x >= 1 && md.sub_y >= 1 && md.sub_z >= 1 && md.sub_x <= 8 && md.sub_y <= 8 && md.sub_z <= 8,
             "subdomain sizes must be in [1, 8]");
  DD_REQUIRE(md.nx % md.sub_x == 0 && md.ny % md.sub_y == 0 && md.nz % md.sub_z == 0,
             "subdomain sizes must divide the mesh");
  // no Dirichlet face: the pure-Neumann problem (semidefinite K, Sect. 2)
  H.neumann = (md.dirichlet_faces & 63u) == 0;
  DD_REQUIRE(!(H.neumann && opt.adaptive), "adaptive constraints are not supported without a Dirichlet face");
  DD_REQUIRE(opt.levels == 2 || opt.levels == 3, "levels must be 2 or 3");
  DD_REQUIRE(opt.weights == DD_WEIGHTS_CARD || opt.weights == DD_WEIGHTS_DIAG, "weights must be card or diag");
  Mesh1& M = H.mesh;
  M.nx = md.nx; M.ny = md.ny; M.nz = md.nz;
  M.sx = md.sub_x; M.sy = md.sub_y; M.sz = md.sub_z;
  M.Sx = M.nx / M.sx; M.Sy = M.ny / M.sy; M.Sz = M.nz / M.sz;
  M.S = M.Sx * M.Sy * M.Sz;
  uint32_t df = md.dirichlet_faces;
  M.fx0 = (df & DD_FACE_X0) ? 1 : 0; M.fx1 = (df & DD_FACE_X1) ? M.nx : M.nx + 1;
  M.fy0 = (df & DD_FACE_Y0) ? 1 : 0; M.fy1 = (df & DD_FACE_Y1) ? M.ny : M.ny + 1;
  M.fz0 = (df & DD_FACE_Z0) ? 1 : 0; M.fz1 = (df & DD_FACE_Z1) ? M.nz : M.nz + 1;
  const int64_t Nfx = M.fx1 - M.fx0, Nfy = M.fy1 - M.fy0, Nfz = M.fz1 - M.fz0;
  DD_REQUIRE(Nfx > 0 && Nfy > 0 && Nfz > 0, "no free nodes");
  M.n_free = Nfx * Nfy * Nfz;
  M.NLx = M.sx + 1; M.NLy = M.sy + 1; M.NLz = M.sz + 1;
  M.NL = M.NLx * M.NLy * M.NLz;
  M.xc.assign(md.xc, md.xc + M.nx + 1);
  M.yc.assign(md.yc, md.yc + M.ny + 1);
  M.zc.assign(md.zc, md.zc + M.nz + 1);
  for (int i = 0; i < M.nx; ++i) DD_REQUIRE(M.xc[i + 1] > M.xc[i], "x coordinates must increase");
  for (int i = 0; i < M.ny; ++i) DD_REQUIRE(M.yc[i + 1] > M.yc[i], "y coordinates must increase");
  for (int i = 0; i < M.nz; ++i) DD_REQUIRE(M.zc[i + 1] > M.zc[i], "z coordinates must increase");
  const int64_t E = (int64_t)M.nx * M.ny * M.nz;
  M.ecx.resize(E); M.ecy.resize(E); M.ecz.resize(E);
  for (int ez = 0; ez < M.nz; ++ez)
    for (int ey = 0; ey < M.ny; ++ey)
      for (int ex = 0; ex < M.nx; ++ex) {
        int64_t e = ex + (int64_t)M.nx * (ey + (int64_t)M.ny * ez);
        double k = md.coef ? md.coef[e] : 1.0;
        DD_REQUIRE(k > 0.0 && std::isfinite(k), "coefficients must be positive and finite");
        double hx = M.xc[ex + 1] - M.xc[ex], hy = M.yc[ey + 1] - M.yc[ey], hz = M.zc[ez + 1] - M.zc[ez];
        M.ecx[e] = k * hy * hz / (36.0 * hx);
        M.ecy[e] = k * hx * hz / (36.0 * hy);
        M.ecz[e] = k * hx * hy / (36.0 * hz);
      }

  // ---- interface numbering (free nodes shared by more than one subdomain) ----
  auto cut = [](int p, int n, int s) { return p % s == 0 && p > 0 && p < n; };
  auto is_free = [&](int x, int y, int z) {
    return x >= M.fx0 && x < M.fx1 && y >= M.fy0 && y < M.fy1 && z >= M.fz0 && z < M.fz1;
  };
  auto free_idx = [&](int x, int y, int z) -> int64_t {
    return (x - M.fx0) + Nfx * ((y - M.fy0) + Nfy * (int64_t)(z - M.fz0));
  };
  std::vector<int> gamma_of_free(M.n_free, -1);
  int64_t nG = 0;
  for (int z = M.fz0; z < M.fz1; ++z)
    for (int y = M.fy0; y < M.fy1; ++y)
      for (int x = M.fx0; x < M.fx1; ++x)
        if (cut(x, M.nx, M.sx) || cut(y, M.ny, M.sy) || cut(z, M.nz, M.sz)) {
          gamma_of_free[free_idx(x, y, z)] = (int)nG++;
          M.gamma_free.push_back(free_idx(x, y, z));
        }
  Level& L1 = H.l1;
  L1.S = M.S;
  L1.n_gamma = nG;
  DD_REQUIRE(nG > 0, "partition has no interface (one subdomain)");
  DD_REQUIRE(M.NL <= 729, "local node grid too large");

  // ---- per-subdomain local numbering ----
  M.lidx.assign((size_t)M.S * M.NL, INT16_MIN);
  L1.goff.assign(M.S + 1, 0);
  L1.ioff.assign(M.S + 1, 0);
  std::vector<std::vector<int>> Iloc(M.S), Gloc(M.S);  // positions in the local free-node list
  std::vector<int> nloc(M.S);
  std::vector<std::vector<int>> lfree(M.S);            // local node id of each local free node
  for (int s = 0; s < M.S; ++s) {
    int I = s % M.Sx, J = (s / M.Sx) % M.Sy, Kk = s / (M.Sx * M.Sy);
    int ni = 0, ng = 0, nl = 0;
    for (int c = 0; c < M.NLz; ++c)
      for (int b = 0; b < M.NLy; ++b)
        for (int a = 0; a < M.NLx; ++a) {
          int x = I * M.sx + a, y = J * M.sy + b, z = Kk * M.sz + c;
          int l = a + M.NLx * (b + M.NLy * c);
          if (!is_free(x, y, z)) continue;
          lfree[s].push_back(l);
          if (gamma_of_free[free_idx(x, y, z)] >= 0) {
            M.lidx[(size_t)s * M.NL + l] = (int16_t)(-1 - ng);
            Gloc[s].push_back(nl);
            L1.gmap.push_back(gamma_of_free[free_idx(x, y, z)]);
            ng++;
          } else {
            M.lidx[(size_t)s * M.NL + l] = (int16_t)ni;
            Iloc[s].push_back(nl);
            ni++;
          }
          nl++;
        }
    nloc[s] = nl;
    L1.goff[s + 1] = L1.goff[s] + ng;
    L1.ioff[s + 1] = L1.ioff[s] + ni;
  }
  build_copy_csr(nG, L1.goff, L1.gmap, L1.gptr, L1.gidx);

  // ---- globs from sharing sets ----
  auto axis_subs = [](int p, int n, int s, int* out) -> int {
    if (p % s == 0 && p > 0 && p < n) { out[0] = p / s - 1; out[1] = p / s; return 2; }
    out[0] = std::min(p / s, n / s - 1);
    return 1;
  };
  Globs gl = make_globs(nG, [&](int64_t g, std::vector<int>& subs) {
    int64_t f = M.gamma_free[g];
    int x = (int)(f % Nfx) + M.fx0, y = (int)((f / Nfx) % Nfy) + M.fy0, z = (int)(f / (Nfx * Nfy)) + M.fz0;
    int ax[2], ay[2], az[2];
    int nxs = axis_subs(x, M.nx, M.sx, ax), nys = axis_subs(y, M.ny, M.sy, ay), nzs = axis_subs(z, M.nz, M.sz, az);
    for (int k = 0; k < nzs; ++k)
      for (int j = 0; j < nys; ++j)
        for (int i = 0; i < nxs; ++i) subs.push_back(ax[i] + M.Sx * (ay[j] + M.Sy * az[k]));
    std::sort(subs.begin(), subs.end());
  });
  std::vector<CoarseDof> cd = select_coarse(gl, opt.use_corners, opt.use_edges, opt.use_faces);
  DD_REQUIRE(!cd.empty(), "no coarse degrees of freedom selected");

  // ---- local stiffness matrices (closed-form Kronecker form of the Q1 brick), built per subdomain ----
  auto kloc_fn = [&](int s, std::vector<double>& K) {
    int I = s % M.Sx, J = (s / M.Sx) % M.Sy, Kk = s / (M.Sx * M.Sy);
    int nl = nloc[s];
    std::vector<int> pos(M.NL, -1);
    for (int t = 0; t < nl; ++t) pos[lfree[s][t]] = t;
    K.assign((size_t)nl * nl, 0.0);
    for (int ec = 0; ec < M.sz; ++ec)
      for (int eb = 0; eb < M.sy; ++eb)
        for (int ea = 0; ea < M.sx; ++ea) {
          int64_t e = (I * M.sx + ea) + (int64_t)M.nx * ((J * M.sy + eb) + (int64_t)M.ny * (Kk * M.sz + ec));
          double cx = M.ecx[e], cy = M.ecy[e], cz = M.ecz[e];
          for (int p = 0; p < 8; ++p) {
            int lp = (ea + (p & 1)) + M.NLx * ((eb + ((p >> 1) & 1)) + M.NLy * (ec + (p >> 2)));
            int ip = pos[lp];
            if (ip < 0) continue;
            for (int q = 0; q < 8; ++q) {
              int lq = (ea + (q & 1)) + M.NLx * ((eb + ((q >> 1) & 1)) + M.NLy * (ec + (q >> 2)));
              int iq = pos[lq];
              if (iq < 0) continue;
              int d = p ^ q;
              double sx = (d & 1) ? -1.0 : 1.0, mx = (d & 1) ? 1.0 : 2.0;
              double sy = (d & 2) ? -1.0 : 1.0, my = (d & 2) ? 1.0 : 2.0;
              double sz = (d & 4) ? -1.0 : 1.0, mz = (d & 4) ? 1.0 : 2.0;
              K[(size_t)ip * nl + iq] += cx * sx * my * mz + cy * mx * sy * mz + cz * mx * my * sz;
            }
          }
        }
  };
  auto kdiag_fn = [&](int s, std::vector<double>& d) {  // diagonal: every corner of a brick adds 4(cx+cy+cz)
    int I = s % M.Sx, J = (s / M.Sx) % M.Sy, Kk = s / (M.Sx * M.Sy);
    int nl = nloc[s];
    std::vector<int> pos(M.NL, -1);
    for (int t = 0; t < nl; ++t) pos[lfree[s][t]] = t;
    d.assign(nl, 0.0);
    for (int ec = 0; ec < M.sz; ++ec)
      for (int eb = 0; eb < M.sy; ++eb)
        for (int ea = 0; ea < M.sx; ++ea) {
          int64_t e = (I * M.sx + ea) + (int64_t)M.nx * ((J * M.sy + eb) + (int64_t)M.ny * (Kk * M.sz + ec));
          double v = 4.0 * (M.ecx[e] + M.ecy[e] + M.ecz[e]);
          for (int p = 0; p < 8; ++p) {
            int lp = (ea + (p & 1)) + M.NLx * ((eb + ((p >> 1) & 1)) + M.NLy * (ec + (p >> 2)));
            if (pos[lp] >= 0) d[pos[lp]] += v;
          }
        }
  };
  AdaptiveOpts ad;
  ad.on = opt.adaptive != 0;
  ad.tau = opt.tau;
  ad.max_per_face = opt.max_eig_per_face > 0 ? opt.max_eig_per_face : 10;
  ad.lobpcg = opt.adaptive_solver == DD_EIG_LOBPCG;
  ad.lobpcg_iters = opt.lobpcg_iters;
  DD_REQUIRE(opt.adaptive_solver == DD_EIG_DENSE || opt.adaptive_solver == DD_EIG_LOBPCG,
             "adaptive_solver must be DENSE or LOBPCG");
  DD_REQUIRE(!ad.lobpcg || (opt.lobpcg_iters >= 1 && opt.max_eig_per_face <= LOBPCG_MAXK),
             "adaptive_solver LOBPCG: lobpcg_iters >= 1 and max_eig_per_face <= 10");
  DD_REQUIRE(!ad.on || opt.tau > 1.0, "adaptive threshold tau must exceed 1");
  finish_level(L1, gl, cd, opt.weights, kloc_fn, kdiag_fn, nloc, Iloc, Gloc, false, ad, "level 1");

  // ---- fast diagonalization of K_II (constant coefficient per subdomain, tensor mesh) ----
  {
    bool constant = true;
    std::vector<double> ksub(M.S, 1.0);
    if (md.coef) {
      for (int s = 0; s < M.S && constant; ++s) {
        int I = s % M.Sx, J = (s / M.Sx) % M.Sy, Kk = s / (M.Sx * M.Sy);
        int64_t e0 = (I * M.sx) + (int64_t)M.nx * ((J * M.sy) + (int64_t)M.ny * (Kk * M.sz));
        ksub[s] = md.coef[e0];
        for (int ec = 0; ec < M.sz && constant; ++ec)
          for (int eb = 0; eb < M.sy && constant; ++eb)
            for (int ea = 0; ea < M.sx; ++ea) {
              int64_t e = (I * M.sx + ea) + (int64_t)M.nx * ((J * M.sy + eb) + (int64_t)M.ny * (Kk * M.sz + ec));
              if (md.coef[e] != ksub[s]) {
                constant = false;
                break;
              }
            }
      }
    }
    DD_REQUIRE(opt.local_solver != DD_LOCAL_FDM || constant,
               "local_solver FDM needs a constant coefficient in every subdomain");
    H.local_solver = (opt.local_solver == DD_LOCAL_DENSE || !constant) ? DD_LOCAL_DENSE : DD_LOCAL_FDM;
    if (H.local_solver == DD_LOCAL_FDM) {
      H.fdm.assign(M.S, FdmSub());
      const int ns[3] = {M.sx, M.sy, M.sz}, nn[3] = {M.nx, M.ny, M.nz};
      const int f0[3] = {M.fx0, M.fy0, M.fz0}, f1[3] = {M.fx1, M.fy1, M.fz1};
      const std::vector<double>* cs[3] = {&M.xc, &M.yc, &M.zc};
      int failed = -1;
#pragma omp parallel for schedule(dynamic, 8)
      for (int s = 0; s < M.S; ++s) {
        const int blk[3] = {s % M.Sx, (s / M.Sx) % M.Sy, s / (M.Sx * M.Sy)};
        FdmSub& F = H.fdm[s];
        std::vector<double> lam[3];
        for (int a = 0; a < 3; ++a) {
          const int sa = ns[a], nl = sa + 1, g0 = blk[a] * sa;
          std::vector<double> K1((size_t)nl * nl, 0.0), M1((size_t)nl * nl, 0.0);
          for (int e = 0; e < sa; ++e) {  // 1D stiffness (1/h)[1 -1; -1 1] and mass h[1/3 1/6; 1/6 1/3]
            double h = (*cs[a])[g0 + e + 1] - (*cs[a])[g0 + e];
            K1[(size_t)e * nl + e] += 1.0 / h;
            K1[(size_t)(e + 1) * nl + e + 1] += 1.0 / h;
            K1[(size_t)e * nl + e + 1] -= 1.0 / h;
            K1[(size_t)(e + 1) * nl + e] -= 1.0 / h;
            M1[(size_t)e * nl + e] += h / 3.0;
            M1[(size_t)(e + 1) * nl + e + 1] += h / 3.0;
            M1[(size_t)e * nl + e + 1] += h / 6.0;
            M1[(size_t)(e + 1) * nl + e] += h / 6.0;
          }
          std::vector<int> P;  // interior positions along this axis: not on a cut plane, not Dirichlet
          for (int p = 0; p < nl; ++p) {
            int g = g0 + p;
            bool cutp = g % sa == 0 && g > 0 && g < nn[a];
            if (!cutp && g >= f0[a] && g < f1[a]) P.push_back(p);
          }
          const int n = (int)P.size();
          F.n[a] = n;
          std::vector<double> Ka((size_t)n * n), Ma((size_t)n * n), Linv((size_t)n * n), C((size_t)n * n),
              T((size_t)n * n), U((size_t)n * n);
          for (int i = 0; i < n; ++i)
            for (int j = 0; j < n; ++j) {
              Ka[(size_t)i * n + j] = K1[(size_t)P[i] * nl + P[j]];
              Ma[(size_t)i * n + j] = M1[(size_t)P[i] * nl + P[j]];
            }
          lam[a].resize(n);
          if (!la::cholesky(n, Ma.data())) {
#pragma omp critical
            failed = s;
            continue;
          }
          la::tri_inv_lower(n, Ma.data(), Linv.data());
          // C = L^{-1} K L^{-T}
          la::gemm_nt(n, n, n, 1.0, Ka.data(), Linv.data(), 0.0, T.data());   // K L^{-T}
          la::gemm_nn(n, n, n, Linv.data(), T.data(), C.data());
          for (int i = 0; i < n; ++i)
            for (int j = 0; j < i; ++j) {
              double v = 0.5 * (C[(size_t)i * n + j] + C[(size_t)j * n + i]);
              C[(size_t)i * n + j] = C[(size_t)j * n + i] = v;
            }
          la::sym_eig(n, C.data(), lam[a].data(), U.data());
          // V = L^{-T} U
          F.V[a].assign((size_t)n * n, 0.0);
          for (int i = 0; i < n; ++i)
            for (int j = 0; j < n; ++j) {
              double sacc = 0.0;
              for (int k2 = i; k2 < n; ++k2) sacc += Linv[(size_t)k2 * n + i] * U[(size_t)k2 * n + j];
              F.V[a][(size_t)i * n + j] = sacc;
            }
        }
        const double k = ksub[s];
        F.Dinv.resize((size_t)F.n[0] * F.n[1] * F.n[2]);
        for (int iz = 0; iz < F.n[2]; ++iz)
          for (int iy = 0; iy < F.n[1]; ++iy)
            for (int ix = 0; ix < F.n[0]; ++ix) {
              double d = k * (lam[0][ix] + lam[1][iy] + lam[2][iz]);
              if (!(d > 0.0)) {
#pragma omp critical
                failed = s;
              }
              F.Dinv[((size_t)iz * F.n[1] + iy) * F.n[0] + ix] = 1.0 / d;
            }
        if ((int64_t)F.Dinv.size() != L1.ioff[s + 1] - L1.ioff[s]) {
#pragma omp critical
          failed = s;
        }
      }
      if (failed >= 0)
        throw Error(DD_SINGULAR_LOCAL, "fast diagonalization failed in subdomain " + std::to_string(failed));
    }
  }

  H.levels = opt.levels;
  // Without a Dirichlet face the coarse matrix is singular in the coarse coordinates of the
  // constant function (all ones: corners and averages of a constant are 1), and the coarse
  // right-hand side of a residual orthogonal to the constants is orthogonal to that vector.
  // The grounded matrix K_C + K_C[0][0] e_0 e_0^T is SPD, and its solution u of a consistent
  // system has u_0 = 0 and solves K_C u = g (multiply by the null vector).
  auto ground = [&](int n, std::vector<double>& KC) {
    if (H.neumann && n > 0) KC[0] += KC[0];
  };
  if (opt.levels == 2) {
    std::vector<double> KC = assemble_coarse(L1);
    ground(L1.n_coarse, KC);
    H.KCinv.resize(KC.size());
    if (!la::spd_inverse(L1.n_coarse, KC.data(), H.KCinv.data()))
      throw Error(DD_SINGULAR_LOCAL, "coarse matrix is not SPD");
  } else {
    // ---- level 2: groups of g^3 subdomains, subdomains acting as elements (Sect. 3.2) ----
    int g = std::max(1, opt.coarse_group);
    int Gx = (M.Sx + g - 1) / g, Gy = (M.Sy + g - 1) / g, Gz = (M.Sz + g - 1) / g;
    int S2 = Gx * Gy * Gz;
    std::vector<std::vector<int>> members(S2);
    for (int s = 0; s < M.S; ++s) {
      int I = s % M.Sx, J = (s / M.Sx) % M.Sy, Kk = s / (M.Sx * M.Sy);
      members[(I / g) + Gx * ((J / g) + Gy * (Kk / g))].push_back(s);
    }
    int nC = L1.n_coarse;
    std::vector<std::vector<int>> groups_of_c(nC);
    std::vector<std::vector<int>> ldofs(S2);
    for (int j = 0; j < S2; ++j) {
      std::vector<int> d;
      for (int s : members[j]) d.insert(d.end(), L1.sub[s].cmap.begin(), L1.sub[s].cmap.end());
      std::sort(d.begin(), d.end());
      d.erase(std::unique(d.begin(), d.end()), d.end());
      ldofs[j] = d;
      for (int c : d) groups_of_c[c].push_back(j);
    }
    Level& L2 = H.l2;
    L2.S = S2;
    std::vector<int> gam2_of_c(nC, -1);
    int64_t nG2 = 0;
    for (int c = 0; c < nC; ++c)
      if (groups_of_c[c].size() >= 2) {
        gam2_of_c[c] = (int)nG2++;
        H.gam2_c.push_back(c);
      }
    L2.n_gamma = nG2;
    DD_REQUIRE(nG2 > 0, "three levels need more than one coarse subdomain");
    std::vector<std::vector<double>> K2(S2);
    std::vector<int> nloc2(S2);
    std::vector<std::vector<int>> I2(S2), G2(S2);
    L2.goff.assign(S2 + 1, 0);
    L2.ioff.assign(S2 + 1, 0);
    for (int j = 0; j < S2; ++j) {
      const auto& d = ldofs[j];
      int n = (int)d.size();
      nloc2[j] = n;
      K2[j].assign((size_t)n * n, 0.0);
      for (int s : members[j]) {
        const DenseSub& ds = L1.sub[s];
        std::vector<int> p(ds.nc);
        for (int a = 0; a < ds.nc; ++a) p[a] = (int)(std::lower_bound(d.begin(), d.end(), ds.cmap[a]) - d.begin());
        for (int a = 0; a < ds.nc; ++a)
          for (int b = 0; b < ds.nc; ++b) K2[j][(size_t)p[a] * n + p[b]] += ds.KC[(size_t)a * ds.nc + b];
      }
      for (int t = 0; t < n; ++t) {
        if (gam2_of_c[d[t]] >= 0) {
          G2[j].push_back(t);
          L2.gmap.push_back(gam2_of_c[d[t]]);
        } else {
          I2[j].push_back(t);
          H.imap2.push_back(d[t]);
        }
      }
      L2.goff[j + 1] = L2.goff[j] + (int64_t)G2[j].size();
      L2.ioff[j + 1] = L2.ioff[j] + (int64_t)I2[j].size();
    }
    build_copy_csr(nG2, L2.goff, L2.gmap, L2.gptr, L2.gidx);
    Globs gl2 = make_globs(nG2, [&](int64_t gg, std::vector<int>& subs) { subs = groups_of_c[H.gam2_c[gg]]; });
    std::vector<CoarseDof> cd2 = select_coarse(gl2, true, true, true);
    DD_REQUIRE(!cd2.empty(), "no level-2 coarse dofs");
    finish_level(
        L2, gl2, cd2, opt.weights, [&](int j, std::vector<double>& K) { K = K2[j]; },
        [&](int j, std::vector<double>& d) {
          d.resize(nloc2[j]);
          for (int t = 0; t < nloc2[j]; ++t) d[t] = K2[j][(size_t)t * nloc2[j] + t];
        },
        nloc2, I2, G2, true, AdaptiveOpts(), "level 2");
    std::vector<double> KC3 = assemble_coarse(L2);
    ground(L2.n_coarse, KC3);
    H.KC3inv.resize(KC3.size());
    if (!la::spd_inverse(L2.n_coarse, KC3.data(), H.KC3inv.data()))
      throw Error(DD_SINGULAR_LOCAL, "level-3 coarse matrix is not SPD");
  }
  H.setup_seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
}

}  // namespace dd
