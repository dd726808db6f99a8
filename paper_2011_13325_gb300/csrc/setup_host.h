// Host setup of the hierarchy (internal to libamg).
#pragma once

#include <stdint.h>

#include <array>
#include <string>
#include <vector>

namespace amgsetup {

struct HostBSR {
  int n_rows = 0, n_cols = 0, br = 0, bc = 0;
  std::vector<int> rowptr, colidx;
  std::vector<double> vals;
};

// Auxiliary topology of one level: vertices, edges (i < j) with k x k edge
// matrices E, vertex matrices M, Dirichlet flags, sorted adjacency.
struct Topo {
  int n = 0, d = 0, k = 0;
  std::vector<double> pos, E, M;
  std::vector<int> ei, ej;
  std::vector<char> dir;
  std::vector<int> adj_ptr, adj_nbr, adj_edge;
  // true when every E and M lives in the displacement block only (finest
  // elasticity level, Thm. deng_elast with M = 0)
  bool rot_free = false;
  void build_adj();
  int edge(int a, int b) const;
};

struct Problem {
  int dim = 0, n_vertices = 0;
  int block = 0;  // dofs per vertex: dim (elasticity; also 0) or 1 (the scalar problem)
  const double *coords = nullptr;
  const uint8_t *dirichlet = nullptr;
  const int32_t *rowptr = nullptr, *colidx = nullptr;
  const double *vals = nullptr;
};

struct SetupParams {
  double sigma = 30.0;
  int delta = 1;
  int passes_first = 5, passes_later = 4;
  double omega = 2.0 / 3.0;
  int cap_S_first = 8, cap_S_later = 6, cap_A = 4;
  int coarse_max = 0;
  double min_ratio = 1.5;
  int max_levels = 16;
  int host_threads = 0;  // OpenMP threads of this call (0: the process default)
  bool scalar_only = false;  // Algorithm 1 with mu_s alone (the paper's scalar runs)
};

// Batched evaluation of the pair measure mu_p (Lemma mu2) of one matching
// pass of Algorithm 1: begin_pass receives the pass's topology and its D-hat
// blocks, evaluate the measures of a batch of pairs.  Each returns 0 or an
// error.
struct PairMeasure {
  virtual ~PairMeasure() {}
  virtual int begin_pass(const Topo &T, const std::vector<double> &Dh, int delta) = 0;
  virtual int evaluate(const std::vector<std::array<int, 2>> &pairs, std::vector<double> &mu) = 0;
};

// Receives the levels as they are built: first(A_0), then for every level
// the prolongation P_l; it must return A_{l+1} = P_l^T A_l P_l on the host.
// A sink with device_stages() true also builds, for the agglomerates of
// Algorithm 1, the coarse edge / vertex matrices (coarse_topology) and the
// smoothed prolongation (prolongation: sets *handled = 1 when it built P
// and next_bad, else the host builds them); each returns 0 or an error.
struct LevelSink {
  virtual ~LevelSink() {}
  virtual int first(const HostBSR &A0) = 0;
  virtual int next(int level, const HostBSR &P, HostBSR &A_next) = 0;
  virtual bool device_stages() const { return false; }
  // an evaluator of mu_p for Algorithm 1 (owned by the sink), or NULL: host
  virtual PairMeasure *pair_measure() { return nullptr; }
  virtual int coarse_topology(int level, const Topo &T, const std::vector<int> &agg, int nc,
                              const std::vector<double> &xc, Topo &out) {
    (void)level; (void)T; (void)agg; (void)nc; (void)xc; (void)out;
    return -1;
  }
  virtual int prolongation(int level, const HostBSR &A, const Topo &T, const std::vector<int> &agg,
                           const std::vector<char> &D, int nc, const std::vector<double> &xc,
                           const std::vector<int> &rowmap, const std::vector<char> &bad, bool first,
                           const SetupParams &prm, HostBSR &P, std::vector<char> &next_bad,
                           int *handled) {
    (void)level; (void)A; (void)T; (void)agg; (void)D; (void)nc; (void)xc; (void)rowmap; (void)bad;
    (void)first; (void)prm; (void)P; (void)next_bad;
    *handled = 0;
    return 0;
  }
};

Topo finest_topology(int d, int n, const double *coords, const uint8_t *dirichlet,
                     const int32_t *rp, const int32_t *ci, const double *vals);
// the scalar problem (1 x 1 blocks; coords hold dim values per vertex)
Topo finest_topology_scalar(int dim, int n, const double *coords, const uint8_t *dirichlet,
                            const int32_t *rp, const int32_t *ci, const double *vals);

int build_levels(const Problem &prob, const SetupParams &prm, LevelSink &sink, std::string &err);

// Distance-1 colouring of the block graph of a matrix pattern (CSR, n rows)
// for the hybrid Gauss-Seidel smoother: greedy in smallest-last order
// (repeatedly remove a remaining row of least degree, ties by the smallest
// index; colour in the reverse of the removals, each row the smallest
// colour no already coloured neighbour holds).  Returns the colour of every
// row; *n_colours the number of colours.
std::vector<int> smallest_last_colouring(int n, const int *rowptr, const int *colidx, int *n_colours);

}  // namespace amgsetup
