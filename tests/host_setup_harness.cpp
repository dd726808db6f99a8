// Test driver for the library's host setup (csrc/setup_host.cpp) without a
// GPU: runs amgsetup::build_levels on a problem read from binary files and
// hands it the coarse matrices A_{l+1} = P_l^T A_l P_l from a plain host
// block product (in place of the library's device Galerkin product), then
// writes the prolongations for the Python test to compare with the oracle.
//
// usage: host_setup_harness <dir> <coarse_max>
//   <dir>/problem.bin: int32 dim, n_vertices, nnzb; float64 coords
//   (n x dim); uint8 dirichlet (n); int32 rowptr (n+1), colidx (nnzb);
//   float64 vals (nnzb x dim x dim)
//   writes <dir>/P.bin: int32 n_levels-1; per level int32 n_rows, n_cols,
//   br, bc, nnzb, rowptr, colidx; float64 vals
//
// usage: host_setup_harness --colour <dir>
//   runs amgsetup::smallest_last_colouring (the hybrid Gauss-Seidel
//   smoother's colouring) on <dir>/pattern.bin: int32 n, nnz, rowptr
//   (n+1), colidx (nnz); writes <dir>/colour.bin: int32 n_colours, colour (n)
#include <stdint.h>
#include <stdio.h>
#include <stdlib.h>

#include <map>
#include <string>
#include <vector>

#include "setup_host.h"

using namespace amgsetup;

template <typename T>
static bool get(FILE *f, std::vector<T> &v, size_t n) {
  v.resize(n);
  return n == 0 || fread(v.data(), sizeof(T), n, f) == n;
}

// A_{l+1} = P^T A P, blocks of every structurally reached coarse pair kept,
// columns ascending (the pattern rule of the device product).
struct HostGalerkinSink : LevelSink {
  HostBSR A;
  std::vector<HostBSR> Ps;
  int first(const HostBSR &A0) override {
    A = A0;
    return 0;
  }
  int next(int, const HostBSR &P, HostBSR &An) override {
    Ps.push_back(P);
    const int kf = A.br, kc = P.bc, nc = P.n_cols;
    std::vector<std::vector<std::pair<int, int>>> Rt(nc);  // coarse row -> (fine row, block)
    for (int r = 0; r < P.n_rows; ++r)
      for (int p = P.rowptr[r]; p < P.rowptr[r + 1]; ++p) Rt[P.colidx[p]].push_back({r, p});
    An = HostBSR();
    An.n_rows = An.n_cols = nc;
    An.br = An.bc = kc;
    An.rowptr.assign(nc + 1, 0);
    std::vector<double> AP((size_t)kf * kc);
    for (int I = 0; I < nc; ++I) {
      std::map<int, std::vector<double>> row;
      for (const auto &ip : Rt[I]) {
        const double *Pi = &P.vals[(size_t)ip.second * kf * kc];
        for (int a = A.rowptr[ip.first]; a < A.rowptr[ip.first + 1]; ++a) {
          const int j = A.colidx[a];
          const double *Aij = &A.vals[(size_t)a * kf * kf];
          for (int b = P.rowptr[j]; b < P.rowptr[j + 1]; ++b) {
            const double *Pj = &P.vals[(size_t)b * kf * kc];
            for (int x = 0; x < kf; ++x)
              for (int y = 0; y < kc; ++y) {
                double s = 0.0;
                for (int z = 0; z < kf; ++z) s += Aij[x * kf + z] * Pj[z * kc + y];
                AP[(size_t)x * kc + y] = s;
              }
            std::vector<double> &blk = row[P.colidx[b]];
            if (blk.empty()) blk.assign((size_t)kc * kc, 0.0);
            for (int x = 0; x < kc; ++x)
              for (int y = 0; y < kc; ++y) {
                double s = 0.0;
                for (int z = 0; z < kf; ++z) s += Pi[z * kc + x] * AP[(size_t)z * kc + y];
                blk[(size_t)x * kc + y] += s;
              }
          }
        }
      }
      for (const auto &kv : row) {
        An.colidx.push_back(kv.first);
        An.vals.insert(An.vals.end(), kv.second.begin(), kv.second.end());
      }
      An.rowptr[I + 1] = (int)An.colidx.size();
    }
    A = An;
    return 0;
  }
};

static int colour_main(const std::string &dir) {
  FILE *f = fopen((dir + "/pattern.bin").c_str(), "rb");
  if (!f) return 3;
  int32_t hdr[2];
  if (fread(hdr, 4, 2, f) != 2) return 3;
  std::vector<int32_t> rowptr, colidx;
  if (!get(f, rowptr, (size_t)hdr[0] + 1) || !get(f, colidx, hdr[1])) return 3;
  fclose(f);
  int nc = 0;
  const std::vector<int> colour = smallest_last_colouring(hdr[0], rowptr.data(), colidx.data(), &nc);
  FILE *o = fopen((dir + "/colour.bin").c_str(), "wb");
  if (!o) return 3;
  const int32_t n_col = nc;
  fwrite(&n_col, 4, 1, o);
  fwrite(colour.data(), 4, colour.size(), o);
  fclose(o);
  return 0;
}

int main(int argc, char **argv) {
  if (argc == 3 && std::string(argv[1]) == "--colour") return colour_main(argv[2]);
  if (argc < 3) {
    fprintf(stderr, "usage: %s <dir> <coarse_max> [passes_first passes_later]\n", argv[0]);
    return 2;
  }
  const std::string dir = argv[1];
  FILE *f = fopen((dir + "/problem.bin").c_str(), "rb");
  if (!f) return 3;
  int32_t hdr[4];
  if (fread(hdr, 4, 4, f) != 4) return 3;
  const int dim = hdr[0], n = hdr[1], nnzb = hdr[2], block = hdr[3];
  std::vector<double> coords, vals;
  std::vector<uint8_t> dirichlet;
  std::vector<int32_t> rowptr, colidx;
  if (!get(f, coords, (size_t)n * dim) || !get(f, dirichlet, n) || !get(f, rowptr, n + 1) ||
      !get(f, colidx, nnzb) || !get(f, vals, (size_t)nnzb * block * block))
    return 3;
  fclose(f);
  Problem pb;
  pb.dim = dim;
  pb.block = block;
  pb.n_vertices = n;
  pb.coords = coords.data();
  pb.dirichlet = dirichlet.data();
  pb.rowptr = rowptr.data();
  pb.colidx = colidx.data();
  pb.vals = vals.data();
  SetupParams prm;
  prm.coarse_max = atoi(argv[2]);
  if (argc > 4) {  // matching passes on the first / later levels
    prm.passes_first = atoi(argv[3]);
    prm.passes_later = atoi(argv[4]);
  }
  if (argc > 7) {  // mu_s alone; row caps of real-matrix rows on the first / later levels
    prm.scalar_only = atoi(argv[5]) != 0;
    prm.cap_S_first = atoi(argv[6]);
    prm.cap_S_later = atoi(argv[7]);
  }
  HostGalerkinSink sink;
  std::string err;
  if (build_levels(pb, prm, sink, err) != 0) {
    fprintf(stderr, "build_levels: %s\n", err.c_str());
    return 1;
  }
  FILE *o = fopen((dir + "/P.bin").c_str(), "wb");
  if (!o) return 3;
  const int32_t np = (int32_t)sink.Ps.size();
  fwrite(&np, 4, 1, o);
  for (const HostBSR &P : sink.Ps) {
    const int32_t h[5] = {P.n_rows, P.n_cols, P.br, P.bc, (int32_t)P.colidx.size()};
    fwrite(h, 4, 5, o);
    fwrite(P.rowptr.data(), 4, P.rowptr.size(), o);
    fwrite(P.colidx.data(), 4, P.colidx.size(), o);
    fwrite(P.vals.data(), 8, P.vals.size(), o);
  }
  fclose(o);
  return 0;
}
