// Host symbolic stage of HIF-DE in 3D with edge skeletonization
// (Section 4.5); the definitions are in symbolic3x.h.
#include "symbolic3x.h"

#include <algorithm>
#include <climits>
#include <cmath>

#include "host_pool.h"

namespace hif {

namespace {

// Nearest of the ascending positions pos to x2: its index and squared
// distance; tie when a second position is as near.
inline void nearest(int64_t x2, const std::vector<int>& pos, int& idx, int64_t& d2, bool& tie) {
  const int j = (int)(std::lower_bound(pos.begin(), pos.end(), (int)x2) - pos.begin());
  const bool lo = j > 0, hi = j < (int)pos.size();
  const int64_t dl = lo ? (x2 - pos[j - 1]) * (x2 - pos[j - 1]) : INT64_MAX;
  const int64_t dh = hi ? (x2 - pos[j]) * (x2 - pos[j]) : INT64_MAX;
  if (dl <= dh) {
    idx = j - 1;
    d2 = dl;
    tie = hi && dl == dh;
  } else {
    idx = j;
    d2 = dh;
    tie = false;
  }
}

}  // namespace

Symbolic3x::Symbolic3x(int n, int leaf, bool implicit_stencil) : n_(n), implicit_(implicit_stencil) {
  L_ = std::max(1, (int)std::lround(std::log2((double)n / leaf)));
  m_ = n >> L_;
  const int e = n - 1;
  N_ = e * e * e;
  active_.assign(N_, 1);
  active_list_.resize(N_);
  for (int i = 0; i < N_; ++i) active_list_[i] = i;
  of_.resize(N_);
  mark_.assign(N_, -1);
  seen_.assign(N_, 0);
  pos_.assign(N_, -1);
}

const std::vector<int>& Symbolic3x::active() {
  if (active_dirty_) {
    active_list_.clear();
    for (int i = 0; i < N_; ++i)
      if (active_[i]) active_list_.push_back(i);
    active_dirty_ = false;
  }
  return active_list_;
}

bool Symbolic3x::voronoi(int g, const std::vector<std::vector<int>>* fams, int nfam, Key& k) const {
  const int e = n_ - 1;
  const int64_t x2[3] = {2 * (int64_t)(g % e + 1), 2 * (int64_t)((g / e) % e + 1), 2 * (int64_t)(g / (e * e) + 1)};
  int64_t best = INT64_MAX;
  int nbest = 0;
  bool best_tie = false;
  for (int f = 0; f < nfam; ++f) {
    int64_t d = 0;
    bool tie = false;
    int idx[3];
    for (int a = 0; a < 3; ++a) {
      int64_t da;
      bool ta;
      nearest(x2[a], fams[f][a], idx[a], da, ta);
      d += da;
      tie |= ta;
    }
    if (d < best) {
      best = d;
      nbest = 1;
      best_tie = tie;
      k.fam = f;
      k.i[0] = idx[0];
      k.i[1] = idx[1];
      k.i[2] = idx[2];
    } else if (d == best) {
      ++nbest;
    }
  }
  return nbest == 1 && !best_tie;
}

std::vector<int> Symbolic3x::neighbors(const std::vector<int>& c) const {
  if (stamp_ > INT_MAX - 4) {
    std::fill(seen_.begin(), seen_.end(), 0);
    std::fill(clique_seen_.begin(), clique_seen_.end(), 0);
    stamp_ = 0;
  }
  stamp_ += 2;
  const int in_c = stamp_ - 1, in_out = stamp_;
  for (int i : c) seen_[i] = in_c;
  std::vector<int> out;
  auto add = [&](int j) {
    if (seen_[j] != in_c && seen_[j] != in_out) {
      seen_[j] = in_out;
      out.push_back(j);
    }
  };
  if (implicit_) {
    const int e = n_ - 1;
    const int step[3] = {1, e, e * e};
    for (int i : c) {
      const int x[3] = {i % e, (i / e) % e, i / (e * e)};
      for (int a = 0; a < 3; ++a) {
        if (x[a] > 0 && active_[i - step[a]]) add(i - step[a]);
        if (x[a] < e - 1 && active_[i + step[a]]) add(i + step[a]);
      }
    }
  }
  // every clique touching c once (a clique holds many members of c)
  for (int i : c)
    for (int id : of_[i]) {
      if (clique_seen_[id] == in_out) continue;
      clique_seen_[id] = in_out;
      const std::vector<int>& m = clique_[id];
      if (m.size() < 2) continue;
      for (int j : m)
        if (active_[j]) add(j);
    }
  std::sort(out.begin(), out.end());
  return out;
}

std::vector<std::vector<int>> Symbolic3x::cells(int l) {
  std::vector<std::vector<int>> out;
  if (l < 0 || l >= L_) return out;
  const int S = m_ << l, K = 1 << (L_ - l);
  std::vector<int> ctr(K);
  for (int j = 0; j < K; ++j) ctr[j] = (2 * j + 1) * S;
  const std::vector<std::vector<int>> fam[1] = {{ctr, ctr, ctr}};
  const std::vector<int>& act = active();
  const int64_t na = (int64_t)act.size();
  std::vector<int> lin(na);
  const int tasks = task_count(na, 1 << 14);
  parallel_tasks(tasks, [&](int t) {
    int64_t lo, hi;
    task_range(na, tasks, t, lo, hi);
    for (int64_t r = lo; r < hi; ++r) {
      Key k;
      lin[r] = voronoi(act[r], fam, 1, k) ? k.i[0] + K * (k.i[1] + K * k.i[2]) : -1;
    }
  });
  // bucket the members by cell (ascending DOF order within a cell)
  const int nc = K * K * K;
  std::vector<int> start(nc + 1, 0);
  for (int64_t r = 0; r < na; ++r)
    if (lin[r] >= 0) ++start[lin[r] + 1];
  for (int c = 0; c < nc; ++c) start[c + 1] += start[c];
  std::vector<int> members(start[nc]);
  {
    std::vector<int> fill(start.begin(), start.end() - 1);
    for (int64_t r = 0; r < na; ++r)
      if (lin[r] >= 0) {
        members[fill[lin[r]]++] = act[r];
        mark_[act[r]] = lin[r];
      }
  }
  // Only a clique whose members start in two or more cells can make a DOF
  // leave (the peel only takes members away): mark those once.
  std::vector<char> mixed(clique_.size(), 0);
  for (size_t id = 0; id < clique_.size(); ++id) {
    int first = -1;
    for (int j : clique_[id]) {
      const int cj = mark_[j];
      if (cj < 0) continue;
      if (first < 0) {
        first = cj;
      } else if (cj != first) {
        mixed[id] = 1;
        break;
      }
    }
  }
  // peel, cell by cell: a DOF coupled to a current member of another cell leaves
  const int e = n_ - 1;
  const int step[3] = {1, e, e * e};
  for (int c = 0; c < nc; ++c) {
    std::vector<int> keep;
    for (int s = start[c]; s < start[c + 1]; ++s) {
      const int i = members[s];
      bool ext = false;
      auto other = [&](int j) { return active_[j] && mark_[j] >= 0 && mark_[j] != c; };
      if (implicit_) {
        const int x[3] = {i % e, (i / e) % e, i / (e * e)};
        for (int a = 0; a < 3 && !ext; ++a)
          ext = (x[a] > 0 && other(i - step[a])) || (x[a] < e - 1 && other(i + step[a]));
      }
      for (size_t k = 0; k < of_[i].size() && !ext; ++k) {
        const int id = of_[i][k];
        if (!mixed[id]) continue;
        for (int j : clique_[id])
          if (other(j)) {
            ext = true;
            break;
          }
      }
      if (ext)
        mark_[i] = -1;
      else
        keep.push_back(i);
    }
    if (!keep.empty()) out.push_back(std::move(keep));
  }
  for (int i : members) mark_[i] = -1;
  return out;
}

std::vector<std::vector<int>> Symbolic3x::groups(int l, int kind) {
  std::vector<std::vector<int>> out;
  if (l < 0 || l >= L_ || (kind != 1 && kind != 2)) return out;
  const int S = m_ << l, K = 1 << (L_ - l);
  std::vector<int> ctr(K), pl(K - 1);
  for (int j = 0; j < K; ++j) ctr[j] = (2 * j + 1) * S;
  for (int j = 0; j < K - 1; ++j) pl[j] = 2 * (j + 1) * S;
  std::vector<std::vector<int>> fam[3];
  for (int f = 0; f < 3; ++f)
    for (int a = 0; a < 3; ++a) {
      const bool plane = kind == 1 ? a == f : a != f;   // faces: normal axis; edges: off-axis
      fam[f].push_back(plane ? pl : ctr);
    }
  // dense code, ascending in (family, x index, y index, z index)
  int64_t base[4] = {0, 0, 0, 0};
  for (int f = 0; f < 3; ++f)
    base[f + 1] = base[f] + (int64_t)fam[f][0].size() * fam[f][1].size() * fam[f][2].size();
  const std::vector<int>& act = active();
  const int64_t na = (int64_t)act.size();
  std::vector<int64_t> code(na);
  const int tasks = task_count(na, 1 << 14);
  parallel_tasks(tasks, [&](int t) {
    int64_t lo, hi;
    task_range(na, tasks, t, lo, hi);
    for (int64_t r = lo; r < hi; ++r) {
      Key k;
      if (!voronoi(act[r], fam, 3, k)) {
        code[r] = -1;
        continue;
      }
      const std::vector<std::vector<int>>& F = fam[k.fam];
      code[r] = base[k.fam] + ((int64_t)k.i[0] * F[1].size() + k.i[1]) * F[2].size() + k.i[2];
    }
  });
  std::vector<int> start(base[3] + 1, 0);
  for (int64_t r = 0; r < na; ++r)
    if (code[r] >= 0) ++start[code[r] + 1];
  for (int64_t c = 0; c < base[3]; ++c) start[c + 1] += start[c];
  for (int64_t c = 0; c < base[3]; ++c)
    if (start[c + 1] > start[c]) out.emplace_back().reserve(start[c + 1] - start[c]);
  std::vector<int> slot(base[3], -1);
  int next = 0;
  for (int64_t c = 0; c < base[3]; ++c)
    if (start[c + 1] > start[c]) slot[c] = next++;
  for (int64_t r = 0; r < na; ++r)
    if (code[r] >= 0) out[slot[code[r]]].push_back(act[r]);
  return out;
}

int Symbolic3x::add_clique(const std::vector<int>& members) {
  const int id = (int)clique_.size();
  clique_.push_back(members);
  clique_live_.push_back(members.empty() ? 0 : 1);
  clique_seen_.push_back(0);
  for (int i : members) of_[i].push_back(id);
  return id;
}

std::vector<int> Symbolic3x::touching(const std::vector<int>& c) const {
  std::vector<int> ids;
  for (int i : c)
    for (int id : of_[i])
      if (clique_live_[id]) ids.push_back(id);
  std::sort(ids.begin(), ids.end());
  ids.erase(std::unique(ids.begin(), ids.end()), ids.end());
  return ids;
}

bool Symbolic3x::gather_plan(const std::vector<std::vector<int>>& keys, const std::vector<std::vector<int>>& order,
                             GatherPlan& out) const {
  out = GatherPlan();
  const size_t nt = std::min(keys.size(), order.size());
  out.start.push_back(0);
  bool ok = true;
  for (size_t t = 0; t < nt && ok; ++t) {
    out.dim.push_back((int)order[t].size());
    for (size_t k = 0; k < order[t].size(); ++k) pos_[order[t][k]] = (int)k;
    for (int id : touching(keys[t])) {
      out.clique.push_back(id);
      out.map_start.push_back((int)out.map.size());
      for (int g : clique_[id]) {
        if (pos_[g] < 0) ok = false;
        out.map.push_back(pos_[g]);
      }
    }
    out.start.push_back((int)out.clique.size());
    for (int g : order[t]) pos_[g] = -1;
  }
  return ok;
}

// Deactivates the DOFs and drops them from their cliques (the others keep
// their order; a clique left empty dies).
void Symbolic3x::remove(const std::vector<int>& dofs) {
  std::vector<int> touched;
  for (int d : dofs) {
    active_[d] = 0;
    for (int id : of_[d]) touched.push_back(id);
    of_[d].clear();
  }
  std::sort(touched.begin(), touched.end());
  touched.erase(std::unique(touched.begin(), touched.end()), touched.end());
  for (int id : touched) {
    std::vector<int>& c = clique_[id];
    c.erase(std::remove_if(c.begin(), c.end(), [&](int j) { return !active_[j]; }), c.end());
    if (c.empty()) {
      std::vector<int>().swap(c);
      clique_live_[id] = 0;
    }
  }
  active_dirty_ = true;
}

int Symbolic3x::eliminate(const std::vector<int>& p) {
  const std::vector<int> q = neighbors(p);
  for (int id : touching(p)) {   // all inside p and q: absorbed by the new clique
    std::vector<int>().swap(clique_[id]);
    clique_live_[id] = 0;
  }
  remove(p);
  return q.empty() ? -1 : add_clique(q);
}

int Symbolic3x::skeletonize(const std::vector<int>& c, const std::vector<int>& s) {
  for (int i : c)
    if (i < 0 || i >= N_ || !active_[i]) return -2;
  if (stamp_ > INT_MAX - 4) {
    std::fill(seen_.begin(), seen_.end(), 0);
    stamp_ = 0;
  }
  stamp_ += 2;
  const int in_c = stamp_ - 1, in_s = stamp_;
  for (int i : c) seen_[i] = in_c;
  for (int i : s) {
    if (i < 0 || i >= N_ || seen_[i] != in_c) return -2;
    seen_[i] = in_s;
  }
  std::vector<int> r;
  for (int i : c)
    if (seen_[i] == in_c) r.push_back(i);
  if (r.empty()) return -1;
  remove(r);
  return s.empty() ? -1 : add_clique(s);
}

}  // namespace hif
