// Host-side set-up of the pressure preconditioner's multigrid hierarchy (the
// V-cycle kernels are in step.cu).  Everything here runs once per flow
// description; the order of every loop is fixed, so the hierarchy, and with
// it every iterate of the solver, is the same from run to run.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

#include "amg.cuh"

namespace rbffd {

namespace {

// Off-diagonal part in CSR (columns sorted) plus the diagonal.
struct HostCsr {
  int64_t n = 0;
  std::vector<int64_t> ptr;
  std::vector<int32_t> col;
  std::vector<double> val;
  std::vector<double> diag;
};

// Weighted graph Laplacian of the kept P-node edges.  Returns an error text or
// an empty string.
std::string edge_graph(int64_t M, int64_t ne, const std::vector<int32_t>& e,
                       const std::vector<double>& x, const std::vector<double>& y,
                       const std::vector<uint8_t>& bc, HostCsr* G) {
  // A Dirichlet P-node (bc == RBFFD_PBC_DIRICHLET, open flows) is eliminated:
  // its edges add their weight to the diagonals of both ends but enter no
  // row as off-diagonal entries, so its own row is diagonal only and its
  // neighbours' rows are strictly diagonally dominant (the graph matrix is
  // then nonsingular, like the pressure system with Dirichlet rows).
  auto dir = [&](int32_t i) { return bc[i] == RBFFD_PBC_DIRICHLET; };
  std::vector<uint8_t> inner(ne), has_in(M, 0);
  std::vector<double> dsum(M, 0.0);
  for (int64_t k = 0; k < ne; ++k) {
    const int32_t a = e[2 * k], b = e[2 * k + 1];
    if (a < 0 || a >= M || b < 0 || b >= M) return "an edge end is not a P-node";
    if (a == b) return "an edge joins a P-node to itself";
    inner[k] = !(bc[a] && bc[b]);
    if (inner[k]) has_in[a] = has_in[b] = 1;
    if (dir(a) || dir(b)) {
      const double dx = x[a] - x[b], dy = y[a] - y[b], d2 = dx * dx + dy * dy;
      if (!(d2 > 0.0)) return "an edge has coincident endpoints";
      dsum[a] += 1.0 / d2;
      dsum[b] += 1.0 / d2;
    }
  }
  std::vector<int64_t> cnt(M + 1, 0);
  auto kept = [&](int64_t k) {
    if (dir(e[2 * k]) || dir(e[2 * k + 1])) return false;
    return inner[k] || !has_in[e[2 * k]] || !has_in[e[2 * k + 1]];
  };
  for (int64_t k = 0; k < ne; ++k)
    if (kept(k)) {
      ++cnt[e[2 * k] + 1];
      ++cnt[e[2 * k + 1] + 1];
    }
  for (int64_t i = 0; i < M; ++i) cnt[i + 1] += cnt[i];
  std::vector<int32_t> col(cnt[M]);
  std::vector<double> w(cnt[M]);
  std::vector<int64_t> cur(cnt.begin(), cnt.end() - 1);
  for (int64_t k = 0; k < ne; ++k) {
    if (!kept(k)) continue;
    const int32_t a = e[2 * k], b = e[2 * k + 1];
    const double dx = x[a] - x[b], dy = y[a] - y[b], d2 = dx * dx + dy * dy;
    if (!(d2 > 0.0)) return "an edge has coincident endpoints";
    col[cur[a]] = b;
    w[cur[a]++] = 1.0 / d2;
    col[cur[b]] = a;
    w[cur[b]++] = 1.0 / d2;
  }
  // sort each row by column and merge repeated edges
  G->n = M;
  G->ptr.assign(M + 1, 0);
  G->col.clear();
  G->val.clear();
  G->diag.assign(M, 0.0);
  std::vector<std::pair<int32_t, double>> row;
  for (int64_t i = 0; i < M; ++i) {
    row.clear();
    for (int64_t p = cnt[i]; p < cnt[i + 1]; ++p) row.emplace_back(col[p], w[p]);
    std::sort(row.begin(), row.end(),
              [](const auto& u, const auto& v) { return u.first < v.first; });
    if (row.empty() && !(dsum[i] > 0.0)) return "a P-node has no edge";
    double s = dsum[i];
    for (size_t q = 0; q < row.size(); ++q) {
      if (q > 0 && row[q].first == row[q - 1].first) {
        G->val.back() -= row[q].second;
      } else {
        G->col.push_back(row[q].first);
        G->val.push_back(-row[q].second);
      }
      s += row[q].second;
    }
    G->diag[i] = s;
    G->ptr[i + 1] = (int64_t)G->col.size();
  }
  return std::string();
}

// Greedy pairwise matching: in row order, an unmatched row takes its
// unmatched neighbour of strongest normalised coupling -a_ij / sqrt(a_ii a_jj),
// the lowest column on ties; a row without one stays alone.  (The raw coupling
// -a_ij would pair large aggregates with each other and strand the small ones
// as singletons, and coarsening would stall after a few levels.)
int32_t pairwise(const HostCsr& A, std::vector<int32_t>* agg) {
  agg->assign(A.n, -1);
  int32_t nc = 0;
  for (int64_t i = 0; i < A.n; ++i) {
    if ((*agg)[i] >= 0) continue;
    int32_t best = -1;
    double bw = 0.0;
    for (int64_t p = A.ptr[i]; p < A.ptr[i + 1]; ++p) {
      const int32_t j = A.col[p];
      if ((*agg)[j] >= 0) continue;
      const double dd = A.diag[i] * A.diag[j];
      const double sij = dd > 0.0 ? -A.val[p] / std::sqrt(dd) : 0.0;
      if (sij > bw) {
        bw = sij;
        best = j;
      }
    }
    (*agg)[i] = nc;
    if (best >= 0) (*agg)[best] = nc;
    ++nc;
  }
  return nc;
}

// Children of each aggregate in row order (counting sort).
void children(const std::vector<int32_t>& agg, int32_t nc, std::vector<int64_t>* cptr,
              std::vector<int32_t>* cidx) {
  cptr->assign(nc + 1, 0);
  for (int32_t a : agg) ++(*cptr)[a + 1];
  for (int32_t I = 0; I < nc; ++I) (*cptr)[I + 1] += (*cptr)[I];
  cidx->resize(agg.size());
  std::vector<int64_t> cur(cptr->begin(), cptr->end() - 1);
  for (size_t i = 0; i < agg.size(); ++i) (*cidx)[cur[agg[i]]++] = (int32_t)i;
}

// C = P^T A P for the piecewise-constant P of `agg`.
void galerkin(const HostCsr& A, const std::vector<int32_t>& agg, int32_t nc, HostCsr* C) {
  std::vector<int64_t> cptr;
  std::vector<int32_t> cidx;
  children(agg, nc, &cptr, &cidx);
  C->n = nc;
  C->ptr.assign(nc + 1, 0);
  C->col.clear();
  C->val.clear();
  C->diag.assign(nc, 0.0);
  std::vector<int64_t> pos(nc, -1);
  std::vector<std::pair<int32_t, double>> row;
  for (int32_t I = 0; I < nc; ++I) {
    row.clear();
    double d = 0.0;
    for (int64_t c = cptr[I]; c < cptr[I + 1]; ++c) {
      const int32_t i = cidx[c];
      d += A.diag[i];
      for (int64_t p = A.ptr[i]; p < A.ptr[i + 1]; ++p) {
        const int32_t J = agg[A.col[p]];
        if (J == I) {
          d += A.val[p];
        } else if (pos[J] < 0) {
          pos[J] = (int64_t)row.size();
          row.emplace_back(J, A.val[p]);
        } else {
          row[pos[J]].second += A.val[p];
        }
      }
    }
    for (auto& rv : row) pos[rv.first] = -1;
    std::sort(row.begin(), row.end(),
              [](const auto& u, const auto& v) { return u.first < v.first; });
    for (auto& rv : row) {
      C->col.push_back(rv.first);
      C->val.push_back(rv.second);
    }
    C->diag[I] = d;
    C->ptr[I + 1] = (int64_t)C->col.size();
  }
}

// B[p][q] = A[old[p]][old[q]] (newidx = inverse of old); columns sorted again.
void permute(const HostCsr& A, const std::vector<int32_t>& old, const std::vector<int32_t>& newidx,
             HostCsr* B) {
  B->n = A.n;
  B->ptr.assign(A.n + 1, 0);
  B->col.clear();
  B->val.clear();
  B->diag.assign(A.n, 0.0);
  std::vector<std::pair<int32_t, double>> row;
  for (int64_t p = 0; p < A.n; ++p) {
    const int32_t i = old[p];
    row.clear();
    for (int64_t k = A.ptr[i]; k < A.ptr[i + 1]; ++k) row.emplace_back(newidx[A.col[k]], A.val[k]);
    std::sort(row.begin(), row.end(),
              [](const auto& u, const auto& v) { return u.first < v.first; });
    for (auto& rv : row) {
      B->col.push_back(rv.first);
      B->val.push_back(rv.second);
    }
    B->diag[p] = A.diag[i];
    B->ptr[p + 1] = (int64_t)B->col.size();
  }
}

// Dense inverse of (A + sigma 1 1^T + eps diag(A)) by Cholesky, row-major.
// sigma lifts the constant null vector of the Laplacian to the mean diagonal;
// eps = 1e-10 keeps the factorisation defined if the graph falls apart.
bool coarse_inverse(const HostCsr& A, std::vector<double>* X, bool singular) {
  const int64_t n = A.n;
  std::vector<double> B(n * n, 0.0);
  double dm = 0.0;
  for (int64_t i = 0; i < n; ++i) dm += A.diag[i];
  dm /= (double)n;
  // a graph Laplacian with zero row sums is singular on the constants: the
  // shift sigma 1 1^T makes it definite; with eliminated Dirichlet nodes it
  // is definite already
  const double sigma = singular ? dm / (double)n : 0.0;
  for (int64_t i = 0; i < n; ++i) {
    for (int64_t j = 0; j < n; ++j) B[i * n + j] = sigma;
    B[i * n + i] += A.diag[i] * (1.0 + 1e-10);
    for (int64_t p = A.ptr[i]; p < A.ptr[i + 1]; ++p) B[i * n + A.col[p]] += A.val[p];
  }
  // lower Cholesky factor in place
  for (int64_t j = 0; j < n; ++j) {
    double d = B[j * n + j];
    for (int64_t k = 0; k < j; ++k) d -= B[j * n + k] * B[j * n + k];
    if (!(d > 0.0)) return false;
    const double ljj = std::sqrt(d);
    B[j * n + j] = ljj;
    for (int64_t i = j + 1; i < n; ++i) {
      double s = B[i * n + j];
      for (int64_t k = 0; k < j; ++k) s -= B[i * n + k] * B[j * n + k];
      B[i * n + j] = s / ljj;
    }
  }
  // W = L^-1 (stored transposed: WT[c][i] = W[i][c]), then X = W^T W
  std::vector<double> WT(n * n, 0.0), t(n);
  for (int64_t c = 0; c < n; ++c) {
    for (int64_t i = 0; i < c; ++i) t[i] = 0.0;
    for (int64_t i = c; i < n; ++i) {
      double s = i == c ? 1.0 : 0.0;
      for (int64_t k = c; k < i; ++k) s -= B[i * n + k] * t[k];
      t[i] = s / B[i * n + i];
    }
    for (int64_t i = 0; i < n; ++i) WT[c * n + i] = t[i];
  }
  X->assign(n * n, 0.0);
  for (int64_t a = 0; a < n; ++a)
    for (int64_t b = a; b < n; ++b) {
      double s = 0.0;
      for (int64_t k = std::max(a, b); k < n; ++k) s += WT[a * n + k] * WT[b * n + k];
      (*X)[a * n + b] = (*X)[b * n + a] = s;
    }
  return true;
}

template <typename T>
int aalloc(rbffd_ctx* ctx, Amg* a, T** out, size_t count) {
  void* p = nullptr;
  int rc = check_cuda(ctx, cudaMalloc(&p, sizeof(T) * (count ? count : 1)), "multigrid alloc");
  if (rc) return rc;
  a->allocs.push_back(p);
  *out = (T*)p;
  return RBFFD_OK;
}

template <typename T>
int upload(rbffd_ctx* ctx, Amg* a, const std::vector<T>& h, T** out, cudaStream_t st) {
  int rc = aalloc(ctx, a, out, h.size());
  if (rc) return rc;
  return check_cuda(ctx, cudaMemcpyAsync(*out, h.data(), sizeof(T) * h.size(),
                                         cudaMemcpyHostToDevice, st),
                    "multigrid upload");
}

template <typename T>
int download(rbffd_ctx* ctx, const T* d, size_t count, std::vector<T>* h, cudaStream_t st) {
  h->resize(count);
  return check_cuda(ctx, cudaMemcpyAsync(h->data(), d, sizeof(T) * count, cudaMemcpyDeviceToHost,
                                         st),
                    "multigrid download");
}

}  // namespace

// Block records (see LevelRec) of level l from its host copies.  aux: the
// level-0 P-node index of each row (l = 0, perm0) or the rows of the finer
// level below each row (l > 0, the finer level's aggregate offsets).
template <int W>
int level_records(rbffd_ctx* ctx, Amg* a, int l, const AmgLevel& g,
                  const std::vector<int32_t>& hidx, const std::vector<float>& hval,
                  const std::vector<float>& hd, const std::vector<float>& hwd,
                  const std::vector<int32_t>& cptr, const std::vector<int32_t>& aux, int64_t nc,
                  cudaStream_t st) {
  const int64_t nrec = (nc + kRecAggs - 1) / kRecAggs;
  std::vector<LevelRec<W>> recs((size_t)nrec);
  for (int64_t b = 0; b < nrec; ++b) {
    LevelRec<W>& R = recs[(size_t)b];
    memset(&R, 0, sizeof(R));
    const int64_t I0 = b * kRecAggs, I1 = std::min<int64_t>(I0 + kRecAggs, nc);
    const int64_t f0 = cptr[I0], f1 = cptr[I1];
    if (f1 - f0 > kRecRows)
      return set_error(ctx, RBFFD_ERR_INVALID_ARG, "multigrid block of %lld rows",
                       (long long)(f1 - f0));
    R.f0 = (int32_t)f0;
    R.nrows = (int32_t)(f1 - f0);
    R.nagg = (int32_t)(I1 - I0);
    for (int64_t I = I0; I <= I1; ++I) R.off[I - I0] = (int32_t)(cptr[I] - f0);
    for (int r = 0; r < kRecRows; ++r) {
      const int64_t i = f0 + r;
      const bool in = i < f1;
      for (int s = 0; s < W; ++s) {
        const bool slot = in && s < g.width;
        R.idx[s * kRecRows + r] = slot ? hidx[(size_t)s * g.ld + i] : (int32_t)f0;
        R.val[s * kRecRows + r] = slot ? hval[(size_t)s * g.ld + i] : 0.f;
      }
      R.diag[r] = in ? hd[i] : 0.f;
      R.wd[r] = in ? hwd[i] : 0.f;
    }
    // aux: nrows entries on level 0, nrows + 1 above it (children of the last row end there)
    const int naux = l == 0 ? R.nrows : R.nrows + 1;
    for (int r = 0; r < naux; ++r) R.aux[r] = aux[(size_t)(f0 + r)];
  }
  std::vector<unsigned char> bytes(sizeof(LevelRec<W>) * (size_t)nrec);
  memcpy(bytes.data(), recs.data(), bytes.size());
  const int rc = upload(ctx, a, bytes, &a->rec[l], st);
  if (rc) return rc;
  a->rec_w[l] = W;
  a->rec_n[l] = nrec;
  return RBFFD_OK;
}

void amg_free(Amg* a) {
  if (!a) return;
  for (void* p : a->allocs) cudaFree(p);
  delete a;
}

int amg_build(rbffd_ctx* ctx, const rbffd_flow& f, const double* diag_a, const double* es,
              Amg** out, cudaStream_t st) {
  *out = nullptr;
  if (!f.p_edges || f.n_edges <= 0 || !f.p_x || !f.p_y)
    return set_error(ctx, RBFFD_ERR_INVALID_ARG,
                     "precond = 1 needs the P-node edges (p_edges, n_edges) and p_x, p_y");
  const int64_t M = f.M;
  std::vector<int32_t> e;
  std::vector<double> x, y;
  std::vector<uint8_t> bc;
  int rc = download(ctx, f.p_edges, (size_t)(2 * f.n_edges), &e, st);
  if (!rc) rc = download(ctx, f.p_x, (size_t)M, &x, st);
  if (!rc) rc = download(ctx, f.p_y, (size_t)M, &y, st);
  if (!rc) rc = download(ctx, f.p_bc, (size_t)M, &bc, st);
  if (!rc) rc = check_cuda(ctx, cudaStreamSynchronize(st), "multigrid download");
  if (rc) return rc;
  std::vector<HostCsr> L(1);
  std::string why = edge_graph(M, f.n_edges, e, x, y, bc, &L[0]);
  if (!why.empty()) return set_error(ctx, RBFFD_ERR_INVALID_ARG, "pressure graph: %s", why.c_str());
  std::vector<std::vector<int32_t>> aggs;
  while (L.back().n > kAmgCoarse && (int)L.size() < kAmgMaxLevels) {
    const HostCsr& A = L.back();
    std::vector<int32_t> a1, a2;
    HostCsr A1, A2;
    const int32_t n1 = pairwise(A, &a1);
    galerkin(A, a1, n1, &A1);
    const int32_t n2 = pairwise(A1, &a2);
    galerkin(A1, a2, n2, &A2);
    if ((double)n2 > 0.85 * (double)A.n) break;  // no longer coarsening
    for (auto& v : a1) v = a2[v];
    aggs.push_back(std::move(a1));
    L.push_back(std::move(A2));
  }
  if (L.back().n > 8 * kAmgCoarse)
    return set_error(ctx, RBFFD_ERR_INVALID_ARG,
                     "pressure graph does not coarsen below %lld nodes (disconnected?)",
                     (long long)L.back().n);
  bool pdir = false;
  for (int64_t i = 0; i < M; ++i) pdir = pdir || bc[i] == RBFFD_PBC_DIRICHLET;
  std::vector<double> Xd;
  if (!coarse_inverse(L.back(), &Xd, !pdir))
    return set_error(ctx, RBFFD_ERR_INVALID_ARG, "coarsest pressure graph matrix is not positive");

  // Nested ordering, coarsest to finest: the coarsest level keeps its order,
  // and each finer level lists its rows aggregate by aggregate in the coarser
  // level's order (rows of one aggregate in their previous order).  Every
  // aggregate's rows are then contiguous (children of coarse row I are rows
  // cptr[I] .. cptr[I+1]-1), so restriction and prolongation touch
  // consecutive rows.
  const int nl = (int)L.size();
  std::vector<std::vector<int32_t>> oldi(nl), newi(nl), cptrs(nl);
  oldi[nl - 1].resize(L[nl - 1].n);
  newi[nl - 1].resize(L[nl - 1].n);
  for (int64_t i = 0; i < L[nl - 1].n; ++i) oldi[nl - 1][i] = newi[nl - 1][i] = (int32_t)i;
  for (int l = nl - 2; l >= 0; --l) {
    const int64_t n = L[l].n;
    const int64_t nc = L[l + 1].n;
    std::vector<int64_t> cnt(nc + 1, 0);
    for (int64_t i = 0; i < n; ++i) ++cnt[newi[l + 1][aggs[l][i]] + 1];
    for (int64_t I = 0; I < nc; ++I) cnt[I + 1] += cnt[I];
    std::vector<int64_t> cur(cnt.begin(), cnt.end() - 1);
    oldi[l].resize(n);
    newi[l].resize(n);
    for (int64_t i = 0; i < n; ++i) {
      const int64_t p = cur[newi[l + 1][aggs[l][i]]]++;
      oldi[l][p] = (int32_t)i;
      newi[l][i] = (int32_t)p;
    }
    cptrs[l].assign(cnt.begin(), cnt.end());
    int cw = 0;
    for (int64_t I = 0; I < nc; ++I) cw = std::max<int>(cw, (int)(cnt[I + 1] - cnt[I]));
    if (cw > 4)  // two pairwise passes make aggregates of at most four rows
      return set_error(ctx, RBFFD_ERR_INVALID_ARG, "multigrid aggregate of %d rows", cw);
  }
  for (int l = 0; l < nl - 1; ++l) {
    HostCsr B;
    permute(L[l], oldi[l], newi[l], &B);
    L[l] = std::move(B);
  }

  Amg* a = new Amg();
  auto fail = [&](int code) {
    amg_free(a);
    return code;
  };
  a->nlev = (int)L.size();
  for (int l = 0; l < a->nlev; ++l) {
    const HostCsr& A = L[l];
    AmgLevel& g = a->lev[l];
    g.n = A.n;
    g.ld = round_up(A.n, 32);
    a->sizes.push_back((int)A.n);
    if ((rc = aalloc(ctx, a, &g.r, g.ld)) || (rc = aalloc(ctx, a, &g.z, g.ld))) return fail(rc);
    if (l == a->nlev - 1) break;
    if ((rc = aalloc(ctx, a, &g.x, g.ld))) return fail(rc);
    int width = 1;
    for (int64_t i = 0; i < A.n; ++i) width = std::max<int>(width, (int)(A.ptr[i + 1] - A.ptr[i]));
    g.width = width;
    std::vector<int32_t> hidx((size_t)width * g.ld);
    std::vector<float> hval((size_t)width * g.ld, 0.f), hd(g.ld, 1.f), hwd(g.ld, 0.f);
    for (int64_t i = 0; i < g.ld; ++i)
      for (int s = 0; s < width; ++s) hidx[s * g.ld + i] = (int32_t)std::min<int64_t>(i, A.n - 1);
    for (int64_t i = 0; i < A.n; ++i) {
      for (int64_t p = A.ptr[i]; p < A.ptr[i + 1]; ++p) {
        const int s = (int)(p - A.ptr[i]);
        hidx[s * g.ld + i] = A.col[p];
        hval[s * g.ld + i] = (float)A.val[p];
      }
      hd[i] = (float)A.diag[i];
      hwd[i] = A.diag[i] > 0.0 ? (float)(kAmgOmega / A.diag[i]) : 0.f;
    }
    if ((rc = upload(ctx, a, hidx, &g.idx, st)) || (rc = upload(ctx, a, hval, &g.val, st)) ||
        (rc = upload(ctx, a, hd, &g.diag, st)) || (rc = upload(ctx, a, hwd, &g.wd, st)) ||
        (rc = upload(ctx, a, cptrs[l], &g.cptr, st)))
      return fail(rc);
    if (width <= 16) {
      const std::vector<int32_t>& aux = l == 0 ? oldi[0] : cptrs[l - 1];
      rc = width <= 8 ? level_records<8>(ctx, a, l, g, hidx, hval, hd, hwd, cptrs[l], aux,
                                         L[l + 1].n, st)
                      : level_records<16>(ctx, a, l, g, hidx, hval, hd, hwd, cptrs[l], aux,
                                          L[l + 1].n, st);
      if (rc) return fail(rc);
    }
  }
  a->nc = L.back().n;
  std::vector<float> hX(Xd.begin(), Xd.end());
  if ((rc = upload(ctx, a, hX, &a->Xc, st))) return fail(rc);
  // level-0 scaling: the scaled pressure rows approximate rows of G divided by diag(G)
  // (stored in the level-0 order: entry p belongs to P-node oldi[0][p])
  std::vector<float> hc(M), hce(M), hcn(M);
  double ces = 0.0;
  for (int64_t p = 0; p < M; ++p) {
    const int32_t i = oldi[0][p];
    const double ci = diag_a[i] != 0.0 ? L[0].diag[p] / diag_a[i] : L[0].diag[p];
    hc[p] = (float)ci;
    hcn[i] = (float)ci;
    hce[p] = (float)(ci * es[i]);
  }
  for (int64_t i = 0; i < M; ++i) {  // in P-node order, like the scalar it normalises
    const int32_t p = newi[0][i];
    ces += (diag_a[i] != 0.0 ? L[0].diag[p] / diag_a[i] : L[0].diag[p]) * es[i];
  }
  if ((rc = upload(ctx, a, oldi[0], &a->perm0, st))) return fail(rc);
  if (pdir) {
    // nonsingular system: no rank-one completion (mu = 0, kap = 0)
    a->inv_ces = 0.0;
    a->inv_R = 0.0;
  } else {
    if (!(ces != 0.0) || !std::isfinite(ces))
      return fail(set_error(ctx, RBFFD_ERR_INVALID_ARG, "pressure rank-one column is zero"));
    a->inv_ces = 1.0 / ces;
    a->inv_R = 1.0 / (double)M;
  }
  if ((rc = upload(ctx, a, hc, &a->c, st)) || (rc = upload(ctx, a, hcn, &a->cnode, st)) ||
      (rc = upload(ctx, a, hce, &a->ce, st)) ||
      (rc = aalloc(ctx, a, &a->zp, M)) || (rc = aalloc(ctx, a, &a->zs, M)) ||
      (rc = aalloc(ctx, a, &a->zpd, M)) || (rc = aalloc(ctx, a, &a->zsd, M)))
    return fail(rc);
  if ((rc = check_cuda(ctx, cudaStreamSynchronize(st), "multigrid upload"))) return fail(rc);
  *out = a;
  return RBFFD_OK;
}

}  // namespace rbffd
