// Inspector: the compression modules of Section 3.1 on the host, in native code.
//
//  * tree construction: a perfect binary tree by median splits, kd (the widest
//    bounding-box dimension; lowest dimension on ties; ties of coordinates by input
//    index) or two-means (along the axis of two mutually far points);
//  * interaction computation: a dual-tree traversal from (root, root) that marks a
//    pair far when it is admissible (Section 2.1) and near when two leaves are not;
//  * low-rank approximation: a nested row interpolative decomposition per node,
//    bottom-up, from a column-pivoted Householder QR of K(R, C)^T whose rank is the
//    number of pivots above tol * |R_11| (the srank tuned to the block accuracy),
//    capped at max_rank.
//
// The dense near blocks and the coupling blocks are not formed here: the loader
// evaluates them on the GPU into the packed arena (hmat_blocks.cu).
#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstring>
#include <new>
#include <numeric>
#include <thread>
#include <vector>

#include "hmat_internal.h"

namespace hmat {
namespace {

constexpr int64_t kExactColumnsMaxN = 4096;

double kernel_value(int kernel, double param, const double* x, const double* y, int d) {
  double r2 = 0.0;
  for (int k = 0; k < d; ++k) {
    const double diff = x[k] - y[k];
    r2 += diff * diff;
  }
  if (kernel == HMAT_KERNEL_GAUSSIAN) return std::exp(-r2 / (2.0 * param * param));
  if (kernel == HMAT_KERNEL_IMQ) return 1.0 / std::sqrt(r2 + param * param);
  return r2 > 0.0 ? 1.0 / std::sqrt(r2) : 0.0;  // 1/r, 0 for coincident points
}

template <class F>
void parallel_for(int64_t n, int threads, F&& f) {
  if (n <= 0) return;
  const int t = (int)std::min<int64_t>(threads, n);
  if (t <= 1) {
    for (int64_t i = 0; i < n; ++i) f(i);
    return;
  }
  std::atomic<int64_t> next(0);
  std::vector<std::thread> pool;
  for (int w = 0; w < t; ++w)
    pool.emplace_back([&]() {
      for (int64_t i; (i = next.fetch_add(1)) < n;) f(i);
    });
  for (auto& th : pool) th.join();
}

uint64_t splitmix64(uint64_t& s) {
  uint64_t z = (s += 0x9E3779B97F4A7C15ull);
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

struct Tree {
  int levels = 0;
  int64_t n_nodes = 0, first_leaf = 0;
  std::vector<int64_t> begin, size, perm;
};

int tree_depth(int64_t n, int64_t leaf) {
  int L = 0;
  while ((n + ((int64_t)1 << L) - 1) / ((int64_t)1 << L) > leaf) ++L;
  return L;
}

double sq_dist(const double* x, const double* y, int d) {
  double s = 0.0;
  for (int k = 0; k < d; ++k) {
    const double diff = x[k] - y[k];
    s += diff * diff;
  }
  return s;
}

// Position (in idx) of the point farthest from y, the smallest input index among ties.
int64_t farthest(const double* X, int d, const int64_t* idx, int64_t nb, const double* y) {
  int64_t best = 0;
  double bd = -1.0;
  for (int64_t i = 0; i < nb; ++i) {
    const double v = sq_dist(X + idx[i] * d, y, d);
    if (v > bd || (v == bd && idx[i] < idx[best])) {
      bd = v;
      best = i;
    }
  }
  return best;
}

// Balanced two-means split order of one node (Section 3.1 names two-means for d > 3
// without an algorithm): p is the point farthest from the node's point of smallest
// input index, q the point farthest from p; points are ordered by their projection
// onto q - p (ties by input index), the first floor(n/2) form the left child.
void two_means_order(const double* X, int d, int64_t* idx, int64_t nb) {
  int64_t a0 = 0;
  for (int64_t i = 1; i < nb; ++i)
    if (idx[i] < idx[a0]) a0 = i;
  const int64_t ip = farthest(X, d, idx, nb, X + idx[a0] * d);
  const double* p = X + idx[ip] * d;
  const int64_t iq = farthest(X, d, idx, nb, p);
  const double* q = X + idx[iq] * d;
  std::vector<std::pair<double, int64_t>> key(nb);
  for (int64_t i = 0; i < nb; ++i) {
    double s = 0.0;
    for (int k = 0; k < d; ++k) s += (X[idx[i] * d + k] - p[k]) * (q[k] - p[k]);
    key[i] = {s, idx[i]};
  }
  std::sort(key.begin(), key.end());
  for (int64_t i = 0; i < nb; ++i) idx[i] = key[i].second;
}

void build_tree(const double* X, int64_t n, int d, int leaf, int tree, int threads, Tree* t) {
  t->levels = tree_depth(n, leaf);
  t->n_nodes = ((int64_t)2 << t->levels) - 1;
  t->first_leaf = ((int64_t)1 << t->levels) - 1;
  t->begin.assign(t->n_nodes, 0);
  t->size.assign(t->n_nodes, 0);
  t->perm.resize(n);
  std::iota(t->perm.begin(), t->perm.end(), 0);
  t->size[0] = n;
  for (int level = 0; level < t->levels; ++level) {
    const int64_t lo = ((int64_t)1 << level) - 1, cnt = (int64_t)1 << level;
    parallel_for(cnt, threads, [&](int64_t k) {
      const int64_t a = lo + k, b0 = t->begin[a], nb = t->size[a];
      int64_t* idx = t->perm.data() + b0;
      const int64_t half = nb / 2;
      t->begin[2 * a + 1] = b0;
      t->size[2 * a + 1] = half;
      t->begin[2 * a + 2] = b0 + half;
      t->size[2 * a + 2] = nb - half;
      if (nb == 0) return;
      if (tree == HMAT_TREE_TWO_MEANS) {
        two_means_order(X, d, idx, nb);
        return;
      }
      int dim = 0;
      double best = -1.0;
      for (int j = 0; j < d; ++j) {
        double mn = INFINITY, mx = -INFINITY;
        for (int64_t i = 0; i < nb; ++i) {
          const double v = X[idx[i] * d + j];
          mn = std::min(mn, v);
          mx = std::max(mx, v);
        }
        if (nb > 0 && mx - mn > best) { best = mx - mn; dim = j; }  // strict: first maximum wins
      }
      std::sort(idx, idx + nb, [&](int64_t p, int64_t q) {
        const double vp = X[p * d + dim], vq = X[q * d + dim];
        return vp < vq || (vp == vq && p < q);
      });
    });
  }
}

// Centroid (mean, accumulated point by point in tree order) and radius per node.
void geometry(const Tree& t, const double* Xt, int d, int threads, std::vector<double>* cent, std::vector<double>* rad) {
  cent->assign(t.n_nodes * d, 0.0);
  rad->assign(t.n_nodes, 0.0);
  parallel_for(t.n_nodes, threads, [&](int64_t a) {
    const int64_t b0 = t.begin[a], nb = t.size[a];
    if (nb == 0) return;
    double* c = cent->data() + a * d;
    for (int64_t i = 0; i < nb; ++i)
      for (int j = 0; j < d; ++j) c[j] += Xt[(b0 + i) * d + j];
    for (int j = 0; j < d; ++j) c[j] /= (double)nb;
    double r = 0.0;
    for (int64_t i = 0; i < nb; ++i) {
      double s = 0.0;
      for (int j = 0; j < d; ++j) {
        const double diff = Xt[(b0 + i) * d + j] - c[j];
        s += diff * diff;
      }
      r = std::max(r, std::sqrt(s));
    }
    (*rad)[a] = r;
  });
}

constexpr int kBudgetNeighbours = 32;

// GOFMM's budget admissibility (the paper's H2-b, Section 4.1; no algorithm given): every
// point votes for the leaves of its kBudgetNeighbours nearest other points (squared
// distances summed over the coordinates in order, ties by index); a leaf is near itself
// and the floor(budget * leaves) leaves with the most votes from its points (ties by
// leaf index), symmetrised. Returns, per level, which node pairs have a near leaf pair
// below them (row-major over the level's nodes).
std::vector<std::vector<uint8_t>> budget_near_below(const Tree& t, const double* Xt, int d, double budget,
                                                    int threads) {
  const int64_t n = t.size[0], nl = (int64_t)1 << t.levels, fl = t.first_leaf;
  const int64_t kk = std::min<int64_t>(kBudgetNeighbours, n - 1);
  std::vector<int64_t> nbr((size_t)std::max<int64_t>(n * kk, 1));
  parallel_for(n, threads, [&](int64_t i) {
    std::vector<std::pair<double, int64_t>> best;  // max-heap of the kk best (distance, index)
    best.reserve((size_t)kk + 1);
    for (int64_t j = 0; j < n; ++j) {
      if (j == i) continue;
      const std::pair<double, int64_t> c{sq_dist(Xt + i * d, Xt + j * d, d), j};
      if ((int64_t)best.size() < kk) {
        best.push_back(c);
        std::push_heap(best.begin(), best.end());
      } else if (kk > 0 && c < best.front()) {
        std::pop_heap(best.begin(), best.end());
        best.back() = c;
        std::push_heap(best.begin(), best.end());
      }
    }
    std::sort_heap(best.begin(), best.end());
    for (int64_t r = 0; r < kk; ++r) nbr[i * kk + r] = best[r].second;
  });
  std::vector<int64_t> leaf_of(n);
  for (int64_t i = 0; i < nl; ++i)
    for (int64_t p = t.begin[fl + i]; p < t.begin[fl + i] + t.size[fl + i]; ++p) leaf_of[p] = i;
  const int64_t keep = (int64_t)std::floor(budget * (double)nl);
  std::vector<uint8_t> near((size_t)(nl * nl), 0);
  for (int64_t i = 0; i < nl; ++i) {
    near[i * nl + i] = 1;
    std::vector<int64_t> votes(nl, 0);
    for (int64_t p = t.begin[fl + i]; p < t.begin[fl + i] + t.size[fl + i]; ++p)
      for (int64_t r = 0; r < kk; ++r) votes[leaf_of[nbr[p * kk + r]]]++;
    votes[i] = 0;
    std::vector<int64_t> cand;
    for (int64_t j = 0; j < nl; ++j)
      if (votes[j] > 0) cand.push_back(j);
    std::stable_sort(cand.begin(), cand.end(), [&](int64_t x, int64_t y) { return votes[x] > votes[y]; });
    for (int64_t c = 0; c < (int64_t)cand.size() && c < keep; ++c) {
      near[i * nl + cand[c]] = 1;
      near[cand[c] * nl + i] = 1;
    }
  }
  std::vector<std::vector<uint8_t>> below(t.levels + 1);
  below[t.levels] = near;
  for (int level = t.levels - 1; level >= 0; --level) {
    const int64_t w = (int64_t)1 << level, wc = 2 * w;
    below[level].assign((size_t)(w * w), 0);
    for (int64_t a = 0; a < wc; ++a)
      for (int64_t b = 0; b < wc; ++b)
        if (below[level + 1][a * wc + b]) below[level][(a / 2) * w + b / 2] = 1;
  }
  return below;
}

void interactions(const Tree& t, const double* Xt, int d, int adm, double eta, int threads,
                  std::vector<std::pair<int64_t, int64_t>>* near, std::vector<std::pair<int64_t, int64_t>>* far) {
  std::vector<std::vector<uint8_t>> below;
  if (adm == HMAT_ADM_BUDGET) below = budget_near_below(t, Xt, d, eta, threads);
  std::vector<double> cent, rad, lo, hi, diam;
  if (adm == HMAT_ADM_GEOMETRIC) geometry(t, Xt, d, threads, &cent, &rad);
  if (adm == HMAT_ADM_TAU) {  // bounding boxes and their diagonals
    lo.assign(t.n_nodes * d, 0.0);
    hi.assign(t.n_nodes * d, 0.0);
    diam.assign(t.n_nodes, 0.0);
    parallel_for(t.n_nodes, threads, [&](int64_t a) {
      const int64_t b0 = t.begin[a], nb = t.size[a];
      if (nb == 0) return;
      for (int j = 0; j < d; ++j) {
        double mn = INFINITY, mx = -INFINITY;
        for (int64_t i = 0; i < nb; ++i) {
          mn = std::min(mn, Xt[(b0 + i) * d + j]);
          mx = std::max(mx, Xt[(b0 + i) * d + j]);
        }
        lo[a * d + j] = mn;
        hi[a * d + j] = mx;
      }
      double s = 0.0;
      for (int j = 0; j < d; ++j) {
        const double ext = hi[a * d + j] - lo[a * d + j];
        s += ext * ext;
      }
      diam[a] = std::sqrt(s);
    });
  }
  auto admissible = [&](int64_t a, int64_t b) {
    if (a == b || adm == HMAT_ADM_NONE) return false;
    if (adm == HMAT_ADM_HSS) return true;
    if (adm == HMAT_ADM_BUDGET) {  // far when no near leaf pair lies below the pair
      int l = 0;
      while (((int64_t)2 << l) - 1 <= a) ++l;
      const int64_t base = ((int64_t)1 << l) - 1, w = (int64_t)1 << l;
      return below[l][(a - base) * w + (b - base)] == 0;
    }
    if (adm == HMAT_ADM_TAU) {  // tau * dist(a, b) > diam(a) + diam(b), dist = the gap between the boxes
      double g2 = 0.0;
      for (int j = 0; j < d; ++j) {
        const double gap = std::max(0.0, std::max(lo[b * d + j] - hi[a * d + j], lo[a * d + j] - hi[b * d + j]));
        g2 += gap * gap;
      }
      return eta * std::sqrt(g2) > diam[a] + diam[b];
    }
    double s = 0.0;
    for (int j = 0; j < d; ++j) {
      const double diff = cent[a * d + j] - cent[b * d + j];
      s += diff * diff;
    }
    return std::sqrt(s) > eta * std::max(rad[a], rad[b]);
  };
  std::vector<std::pair<int64_t, int64_t>> frontier{{0, 0}}, next;
  for (int level = 0; level <= t.levels; ++level) {
    next.clear();
    for (auto [a, b] : frontier) {
      if (admissible(a, b)) far->push_back({a, b});
      else if (level == t.levels) near->push_back({a, b});
      else
        for (int64_t ca : {2 * a + 1, 2 * a + 2})
          for (int64_t cb : {2 * b + 1, 2 * b + 2}) next.push_back({ca, cb});
    }
    frontier.swap(next);
  }
  std::sort(near->begin(), near->end());
  std::sort(far->begin(), far->end());
}

// Row ID of M = K(rows, cols) (|rows| x |cols|): M ~= P M[skel, :], from a column-
// pivoted Householder QR of A = M^T (|cols| x |rows|, column-major) stopped at the
// first pivot |R_kk| <= tol |R_11| or at max_rank. P is |rows| x k row-major.
void row_id(const std::vector<double>& Xt, int d, int kernel, double param, const std::vector<int64_t>& rows,
            const std::vector<int64_t>& cols, double tol, int max_rank, std::vector<int64_t>* skel,
            std::vector<double>* P) {
  const int64_t n = (int64_t)rows.size(), m = (int64_t)cols.size();
  skel->clear();
  P->clear();
  if (n == 0 || m == 0) return;
  std::vector<double> A((size_t)(m * n));
  for (int64_t j = 0; j < n; ++j)
    for (int64_t i = 0; i < m; ++i)
      A[j * m + i] = kernel_value(kernel, param, &Xt[cols[i] * d], &Xt[rows[j] * d], d);
  std::vector<int64_t> piv(n);
  std::iota(piv.begin(), piv.end(), 0);
  std::vector<double> vn1(n), vn2(n);
  for (int64_t j = 0; j < n; ++j) {
    double s = 0.0;
    for (int64_t i = 0; i < m; ++i) s += A[j * m + i] * A[j * m + i];
    vn1[j] = vn2[j] = std::sqrt(s);
  }
  const double tol3z = std::sqrt(2.220446049250313e-16);
  const int64_t kmax = std::min<int64_t>({(int64_t)max_rank, n, m});
  double r11 = 0.0;
  int64_t k = 0;
  for (; k < kmax; ++k) {
    int64_t p = k;
    for (int64_t j = k + 1; j < n; ++j)
      if (vn1[j] > vn1[p]) p = j;
    if (p != k) {
      std::swap_ranges(A.begin() + p * m, A.begin() + (p + 1) * m, A.begin() + k * m);
      std::swap(piv[p], piv[k]);
      vn1[p] = vn1[k];
      vn2[p] = vn2[k];
    }
    // Householder reflector of A[k:m, k]
    double* col = &A[k * m];
    const double alpha = col[k];
    double xn = 0.0;
    for (int64_t i = k + 1; i < m; ++i) xn += col[i] * col[i];
    xn = std::sqrt(xn);
    double beta = alpha, tau = 0.0;
    if (xn != 0.0) {
      beta = -std::copysign(std::hypot(alpha, xn), alpha);
      tau = (beta - alpha) / beta;
      const double scal = 1.0 / (alpha - beta);
      for (int64_t i = k + 1; i < m; ++i) col[i] *= scal;
    }
    col[k] = beta;
    const double rkk = std::fabs(beta);
    if (k == 0) r11 = rkk;
    if (!(rkk > tol * r11) || r11 == 0.0) break;  // this pivot is below the accuracy: rank = k
    // apply (I - tau v v^T), v = [1; col[k+1:m]], to the remaining columns
    if (tau != 0.0)
      for (int64_t j = k + 1; j < n; ++j) {
        double* cj = &A[j * m];
        double w = cj[k];
        for (int64_t i = k + 1; i < m; ++i) w += col[i] * cj[i];
        w *= tau;
        cj[k] -= w;
        for (int64_t i = k + 1; i < m; ++i) cj[i] -= w * col[i];
      }
    // downdate the partial column norms (recompute when cancellation is large)
    for (int64_t j = k + 1; j < n; ++j) {
      if (vn1[j] == 0.0) continue;
      const double r = std::fabs(A[j * m + k]) / vn1[j];
      const double temp = std::max(0.0, (1.0 + r) * (1.0 - r));
      const double ratio = vn1[j] / vn2[j];
      if (temp * ratio * ratio <= tol3z) {
        double s = 0.0;
        for (int64_t i = k + 1; i < m; ++i) s += A[j * m + i] * A[j * m + i];
        vn1[j] = vn2[j] = std::sqrt(s);
      } else {
        vn1[j] *= std::sqrt(temp);
      }
    }
  }
  // T = R11^{-1} R12 (k x (n - k)), back substitution column by column
  const int64_t nt = n - k;
  std::vector<double> T((size_t)(k * nt));
  for (int64_t c = 0; c < nt; ++c) {
    for (int64_t i = k - 1; i >= 0; --i) {
      double s = A[(k + c) * m + i];
      for (int64_t j = i + 1; j < k; ++j) s -= A[j * m + i] * T[j * nt + c];
      T[i * nt + c] = s / A[i * m + i];
    }
  }
  P->assign((size_t)(n * k), 0.0);
  skel->resize(k);
  for (int64_t j = 0; j < k; ++j) {
    (*P)[piv[j] * k + j] = 1.0;
    (*skel)[j] = rows[piv[j]];
  }
  for (int64_t c = 0; c < nt; ++c)
    for (int64_t j = 0; j < k; ++j) (*P)[piv[k + c] * k + j] = T[j * nt + c];
}

}  // namespace
}  // namespace hmat

using namespace hmat;

// Inspector-p1 of Section 3.2 ("Reusing inspection"): everything that depends on the
// points and the admissibility only, kept so that a change of kernel or accuracy
// recompresses without rebuilding it.
struct hmat_plan {
  int64_t n = 0;
  int d = 0;
  int threads = 1;
  Tree t;
  std::vector<double> Xt;                           // points in tree order
  std::vector<std::pair<int64_t, int64_t>> near, far;
  std::vector<std::vector<int64_t>> far_of;         // far partners per node
  std::vector<uint8_t> needs;                       // node needs a basis
};

namespace {

bool valid_compress(const hmat_compress_params* c) {
  return c && c->max_rank >= 1 && c->tol >= 0.0 &&
         (c->kernel == HMAT_KERNEL_GAUSSIAN || c->kernel == HMAT_KERNEL_IMQ || c->kernel == HMAT_KERNEL_INVDIST) &&
         (c->kernel == HMAT_KERNEL_INVDIST || c->kernel_param > 0.0);
}

}  // namespace

extern "C" hmat_status hmat_plan_create(const hmat_plan_params* p, hmat_plan_t* out) {
  if (!out) return HMAT_EINVAL;
  *out = nullptr;
  if (!p || p->n_points < 1 || p->dim < 1 || p->dim > 64 || !p->points || p->leaf_size < 2 ||
      (p->admissibility != HMAT_ADM_HSS && p->admissibility != HMAT_ADM_GEOMETRIC &&
       p->admissibility != HMAT_ADM_NONE && p->admissibility != HMAT_ADM_TAU && p->admissibility != HMAT_ADM_BUDGET) ||
      ((p->admissibility == HMAT_ADM_GEOMETRIC || p->admissibility == HMAT_ADM_TAU) && !(p->eta > 0.0)) ||
      (p->admissibility == HMAT_ADM_BUDGET && !(p->eta >= 0.0 && p->eta <= 1.0)) ||
      (p->tree != HMAT_TREE_KD && p->tree != HMAT_TREE_TWO_MEANS))
    return HMAT_EINVAL;
  const int64_t n = p->n_points;
  const int d = p->dim;
  for (int64_t i = 0; i < n * d; ++i)
    if (!std::isfinite(p->points[i])) return HMAT_EINVAL;
  hmat_plan* pl = new (std::nothrow) hmat_plan();
  if (!pl) return HMAT_ENOMEM;
  pl->n = n;
  pl->d = d;
  pl->threads = p->threads > 0 ? p->threads : (int)std::max(1u, std::thread::hardware_concurrency());
  Tree& t = pl->t;
  build_tree(p->points, n, d, p->leaf_size, p->tree, pl->threads, &t);
  pl->Xt.resize((size_t)(n * d));
  for (int64_t k = 0; k < n; ++k) std::memcpy(&pl->Xt[k * d], &p->points[t.perm[k] * d], d * sizeof(double));
  interactions(t, pl->Xt.data(), d, p->admissibility, p->eta, pl->threads, &pl->near, &pl->far);
  pl->far_of.assign(t.n_nodes, {});
  for (auto [a, b] : pl->far) pl->far_of[a].push_back(b);
  pl->needs.assign(t.n_nodes, 0);
  for (int64_t a = 1; a < t.n_nodes; ++a) pl->needs[a] = !pl->far_of[a].empty() || pl->needs[(a - 1) / 2];
  *out = pl;
  return HMAT_OK;
}

extern "C" hmat_status hmat_plan_free(hmat_plan_t plan) {
  delete plan;
  return HMAT_OK;
}

// Inspector-p2: the nested row IDs for this kernel and accuracy, then the load (near
// and coupling blocks evaluated on the GPU).
namespace {

// The row IDs of every node of one level on the GPU; fills skel, basis and rank of
// those nodes from the device's pivots and T = R_11^{-1} R_12.
hmat_status row_ids_gpu(const hmat_plan& pl, const hmat_compress_params& c, const double* d_pts,
                        const std::vector<int64_t>& nodes, const std::vector<std::vector<int64_t>>& rows_of,
                        const std::vector<std::vector<int64_t>>& cols_of, std::vector<std::vector<int64_t>>* skel,
                        std::vector<std::vector<double>>* basis, std::vector<int32_t>* rank) {
  const int64_t nj = (int64_t)nodes.size();
  if (nj == 0) return HMAT_OK;
  std::vector<IdJob> jobs(nj);
  std::vector<int64_t> ids;
  int64_t a_total = 0, piv_total = 0, max_rows = 1;
  for (int64_t t = 0; t < nj; ++t) {
    const auto& r = rows_of[t];
    const auto& cc = cols_of[t];
    jobs[t] = IdJob{a_total, (int64_t)ids.size(), (int64_t)(ids.size() + r.size()), piv_total, (int32_t)r.size(),
                    (int32_t)cc.size()};
    ids.insert(ids.end(), r.begin(), r.end());
    ids.insert(ids.end(), cc.begin(), cc.end());
    a_total += (int64_t)r.size() * (int64_t)cc.size();
    piv_total += (int64_t)r.size();
    max_rows = std::max<int64_t>(max_rows, (int64_t)r.size());
  }
  IdJob* d_jobs = nullptr;
  int64_t* d_ids = nullptr;
  double* d_work = nullptr;
  int32_t* d_piv = nullptr;
  int32_t* d_rank = nullptr;
  auto release = [&]() {
    cudaFree(d_jobs);
    cudaFree(d_ids);
    cudaFree(d_work);
    cudaFree(d_piv);
    cudaFree(d_rank);
  };
  cudaError_t e = cudaMalloc((void**)&d_jobs, sizeof(IdJob) * nj);
  if (e == cudaSuccess) e = cudaMalloc((void**)&d_ids, sizeof(int64_t) * std::max<size_t>(ids.size(), 1));
  if (e == cudaSuccess) e = cudaMalloc((void**)&d_work, sizeof(double) * std::max<int64_t>(a_total, 1));
  if (e == cudaSuccess) e = cudaMalloc((void**)&d_piv, sizeof(int32_t) * std::max<int64_t>(piv_total, 1));
  if (e == cudaSuccess) e = cudaMalloc((void**)&d_rank, sizeof(int32_t) * nj);
  if (e == cudaSuccess) e = cudaMemcpy(d_jobs, jobs.data(), sizeof(IdJob) * nj, cudaMemcpyHostToDevice);
  if (e == cudaSuccess && !ids.empty())
    e = cudaMemcpy(d_ids, ids.data(), sizeof(int64_t) * ids.size(), cudaMemcpyHostToDevice);
  if (e == cudaSuccess)
    e = launch_row_id(d_jobs, nj, max_rows, d_pts, pl.d, d_ids, c.kernel, c.kernel_param, c.tol, c.max_rank, d_work,
                      d_piv, d_rank, 0);
  if (e == cudaSuccess) e = cudaDeviceSynchronize();
  std::vector<int32_t> rk(nj), piv(std::max<int64_t>(piv_total, 1));
  if (e == cudaSuccess) e = cudaMemcpy(rk.data(), d_rank, sizeof(int32_t) * nj, cudaMemcpyDeviceToHost);
  if (e == cudaSuccess) e = cudaMemcpy(piv.data(), d_piv, sizeof(int32_t) * piv.size(), cudaMemcpyDeviceToHost);
  std::vector<double> T;
  for (int64_t t = 0; t < nj && e == cudaSuccess; ++t) {
    const int64_t a = nodes[t], n = jobs[t].n_rows, m = jobs[t].n_cols, k = rk[t];
    const int32_t* pv = piv.data() + jobs[t].piv_off;
    // T (k x (n - k)): rows 0..k-1 of the columns k..n-1 of this node's A
    T.assign((size_t)(k * (n - k)), 0.0);
    if (k > 0 && n > k)
      e = cudaMemcpy2D(T.data(), (size_t)k * sizeof(double), d_work + jobs[t].a_off + k * m, (size_t)m * sizeof(double),
                       (size_t)k * sizeof(double), (size_t)(n - k), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) break;
    auto& P = (*basis)[a];
    P.assign((size_t)(n * k), 0.0);
    (*skel)[a].resize(k);
    for (int64_t j = 0; j < k; ++j) {
      P[pv[j] * k + j] = 1.0;
      (*skel)[a][j] = rows_of[t][pv[j]];
    }
    for (int64_t cix = 0; cix < n - k; ++cix)
      for (int64_t j = 0; j < k; ++j) P[pv[k + cix] * k + j] = T[cix * k + j];
    (*rank)[a] = (int32_t)k;
  }
  release();
  if (e != cudaSuccess) {
    cudaGetLastError();
    return cuda_status(e);
  }
  return HMAT_OK;
}

}  // namespace

extern "C" hmat_status hmat_plan_build(hmat_plan_t pl, const hmat_compress_params* c, int flags, hmat_t* out) {
  if (!out) return HMAT_EINVAL;
  *out = nullptr;
  if (flags & ~(HMAT_LOAD_MIXED | HMAT_LOAD_MIXED_ONLY | HMAT_BUILD_ID_GPU | HMAT_BUILD_NEAR_OTF))
    return HMAT_EUNSUPPORTED;
  if ((flags & HMAT_BUILD_NEAR_OTF) && (flags & (HMAT_LOAD_MIXED | HMAT_LOAD_MIXED_ONLY))) return HMAT_EUNSUPPORTED;
  if (!pl || !valid_compress(c)) return HMAT_EINVAL;
  const Tree& t = pl->t;
  const int64_t n = pl->n;
  const int d = pl->d;
  const int threads = pl->threads;
  const std::vector<double>& Xt = pl->Xt;
  const bool exact = c->exact_columns > 0 || (c->exact_columns < 0 && n <= kExactColumnsMaxN);
  const int64_t n_sample = std::max<int64_t>(4 * (int64_t)c->max_rank, 512);
  std::vector<std::vector<int64_t>> skel(t.n_nodes);
  std::vector<std::vector<double>> basis(t.n_nodes);
  std::vector<int32_t> rank(t.n_nodes, 0);
  const bool on_gpu = (flags & HMAT_BUILD_ID_GPU) != 0;
  double* d_pts = nullptr;
  if (on_gpu) {
    cudaError_t e = cudaMalloc((void**)&d_pts, sizeof(double) * std::max<size_t>(Xt.size(), 1));
    if (e == cudaSuccess) e = cudaMemcpy(d_pts, Xt.data(), sizeof(double) * Xt.size(), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) {
      cudaFree(d_pts);
      cudaGetLastError();
      return cuda_status(e);
    }
  }
  for (int level = t.levels; level >= 1; --level) {
    const int64_t lo = ((int64_t)1 << level) - 1, cnt = (int64_t)1 << level;
    std::vector<std::vector<int64_t>> rows_of(on_gpu ? cnt : 0), cols_of(on_gpu ? cnt : 0);
    parallel_for(cnt, threads, [&](int64_t k) {
      const int64_t a = lo + k;
      if (!pl->needs[a]) return;
      std::vector<int64_t> rows;
      if (level == t.levels) {
        rows.resize(t.size[a]);
        std::iota(rows.begin(), rows.end(), t.begin[a]);
      } else {
        rows = skel[2 * a + 1];
        rows.insert(rows.end(), skel[2 * a + 2].begin(), skel[2 * a + 2].end());
      }
      std::vector<int64_t> cols;
      for (int64_t g = a;; g = (g - 1) / 2) {
        for (int64_t b : pl->far_of[g])
          for (int64_t i = 0; i < t.size[b]; ++i) cols.push_back(t.begin[b] + i);
        if (g == 0) break;
      }
      std::sort(cols.begin(), cols.end());
      if (!exact && (int64_t)cols.size() > n_sample) {  // seeded uniform sample without replacement
        uint64_t state = c->sample_seed * 0x100000001B3ull + (uint64_t)a;
        for (int64_t i = 0; i < n_sample; ++i) {
          const int64_t j = i + (int64_t)(splitmix64(state) % (uint64_t)(cols.size() - i));
          std::swap(cols[i], cols[j]);
        }
        cols.resize(n_sample);
        std::sort(cols.begin(), cols.end());
      }
      if (on_gpu) {
        rows_of[k] = std::move(rows);
        cols_of[k] = std::move(cols);
        return;
      }
      row_id(Xt, d, c->kernel, c->kernel_param, rows, cols, c->tol, c->max_rank, &skel[a], &basis[a]);
      rank[a] = (int32_t)skel[a].size();
    });
    if (on_gpu) {
      std::vector<int64_t> nodes;
      std::vector<std::vector<int64_t>> r2, c2;
      for (int64_t k = 0; k < cnt; ++k)
        if (pl->needs[lo + k]) {
          nodes.push_back(lo + k);
          r2.push_back(std::move(rows_of[k]));
          c2.push_back(std::move(cols_of[k]));
        }
      const hmat_status st = row_ids_gpu(*pl, *c, d_pts, nodes, r2, c2, &skel, &basis, &rank);
      if (st != HMAT_OK) {
        cudaFree(d_pts);
        return st;
      }
    }
  }
  cudaFree(d_pts);

  // assemble the hmat_desc structure (blocks are evaluated on the device)
  std::vector<int64_t> near_ptr(t.first_leaf + 2, 0), far_ptr(t.n_nodes + 1, 0);
  std::vector<int32_t> near_idx, far_idx;
  for (auto [i, j] : pl->near) near_ptr[i - t.first_leaf + 1]++;
  for (size_t i = 1; i < near_ptr.size(); ++i) near_ptr[i] += near_ptr[i - 1];
  for (auto [i, j] : pl->near) near_idx.push_back((int32_t)(j - t.first_leaf));
  for (auto [a, b] : pl->far) far_ptr[a + 1]++;
  for (size_t i = 1; i < far_ptr.size(); ++i) far_ptr[i] += far_ptr[i - 1];
  for (auto [a, b] : pl->far) far_idx.push_back((int32_t)b);
  std::vector<const double*> basis_ptr(t.n_nodes, nullptr);
  std::vector<int64_t> skel_points;
  for (int64_t a = 0; a < t.n_nodes; ++a) {
    if (rank[a] > 0) basis_ptr[a] = basis[a].data();
    skel_points.insert(skel_points.end(), skel[a].begin(), skel[a].end());
  }
  hmat_desc desc;
  desc.n_points = n;
  desc.levels = t.levels;
  desc.node_begin = t.begin.data();
  desc.node_size = t.size.data();
  desc.rank = rank.data();
  desc.near_ptr = near_ptr.data();
  desc.near_idx = near_idx.data();
  desc.far_ptr = far_ptr.data();
  desc.far_idx = far_idx.data();
  desc.basis = basis_ptr.data();
  desc.coupling = nullptr;
  desc.near = nullptr;
  desc.perm = t.perm.data();
  DeviceBlockSource src{Xt.data(), d, skel_points.data(), c->kernel, c->kernel_param};
  return load_impl(&desc, &src, flags & (HMAT_LOAD_MIXED | HMAT_LOAD_MIXED_ONLY | HMAT_BUILD_NEAR_OTF), out);
}

extern "C" hmat_status hmat_build(const hmat_build_params* p, int flags, hmat_t* out) {
  if (!out) return HMAT_EINVAL;
  *out = nullptr;
  if (flags & ~(HMAT_LOAD_MIXED | HMAT_LOAD_MIXED_ONLY | HMAT_BUILD_ID_GPU | HMAT_BUILD_NEAR_OTF))
    return HMAT_EUNSUPPORTED;
  if ((flags & HMAT_BUILD_NEAR_OTF) && (flags & (HMAT_LOAD_MIXED | HMAT_LOAD_MIXED_ONLY))) return HMAT_EUNSUPPORTED;
  if (!p) return HMAT_EINVAL;
  const hmat_compress_params c{p->kernel, p->kernel_param, p->tol, p->max_rank, p->exact_columns, p->sample_seed};
  if (!valid_compress(&c)) return HMAT_EINVAL;
  const hmat_plan_params pp{p->n_points, p->dim, p->points, p->admissibility, p->eta, p->leaf_size, p->threads,
                            p->tree};
  hmat_plan_t plan = nullptr;
  hmat_status st = hmat_plan_create(&pp, &plan);
  if (st != HMAT_OK) return st;
  st = hmat_plan_build(plan, &c, flags, out);
  hmat_plan_free(plan);
  return st;
}
