// Host-side plan of the DKHn transformation with the exponential parametrisation (Sec. II.C):
// the list of matrix operations that builds the terms of the transformed Hamiltonian and the
// anti-Hermitian generators W_k, as products of n x n (two-component: quaternion) matrices
// that the device then executes in order.  Plain C++ (no CUDA), so it is also compiled and
// checked on the host.
//
// The free-particle transformed Hamiltonian is H^0 = E0 + E1 + O1 (E even, O odd, subscript =
// order in the potential).  Step k applies exp(W_k) . exp(-W_k), expanded as
// sum_j ad_{W_k}^j / j! and cut at order n, with W_k chosen so that [W_k, E0] = -O_k removes
// the odd term of order k: (W_k)_ij = (O_k)_ij / (E0_i + E0_j), no product.  Terms are kept per
// (order, parity) and only the blocks a later step or the final Hamiltonian reads are formed:
//   [W, odd X]  is even: upper block  W X+ + (W X+)+  (one product),
//                        lower block -(W+ X + (W+ X)+) (one product, only when needed);
//   [W, even X] is odd:  block W X' - X W (two products; X' the lower block of X);
//   ad_{W_k}(E0) = -O_k, so ad^j(E0) = -ad^(j-1)(O_k) reuses the chain of O_k.
// The final DKHn Hamiltonian is E0 - c^2 + sum_{l<=n} (E_l upper block) after the steps
// k <= n/2 (later steps only change orders above n).  The number of products this plan needs
// is the P(n) of the paper's Table I ("this work" column).
#pragma once

#include <map>
#include <utility>
#include <vector>

namespace x2c {
namespace dkh {

enum Part { kUpper = 0, kLower = 1, kOdd = 2 };
enum OpType { kGemm = 0, kHerm = 1, kKin = 2, kLin = 3 };

// One device operation on slots (each slot: one n x n quaternion matrix per problem).
struct Op {
  int type;
  int dst;
  int a = -1, b = -1;         // kGemm: dst = alpha op(a) op(b) + beta dst;  kHerm/kKin: source a
  bool adj_a = false, adj_b = false;
  double alpha = 1.0, beta = 0.0;
  std::vector<std::pair<double, int>> lin;  // kLin: dst = sum coef * slot
};

struct Node {
  int order = 0;
  bool even = true;
  int kind = 0;  // 0 given (leaf), 1 sum, 2 commutator [W, X], 3 generator W from an odd term
  std::vector<std::pair<double, int>> terms;
  int W = -1, X = -1, src = -1;
  int slot[3] = {-1, -1, -1};
};

class Plan {
 public:
  // Leaf slots: 0 = E1 (upper), 1 = E1' (lower), 2 = O1.
  static constexpr int kSlotE1 = 0, kSlotE1p = 1, kSlotO1 = 2;

  explicit Plan(int order) : n_(order) {
    Node e1;
    e1.order = 1;
    e1.even = true;
    e1.slot[kUpper] = kSlotE1;
    e1.slot[kLower] = kSlotE1p;
    Node o1;
    o1.order = 1;
    o1.even = false;
    o1.slot[kOdd] = kSlotO1;
    nodes_.push_back(e1);
    nodes_.push_back(o1);
    H_[{1, 1}] = 0;
    H_[{1, 0}] = 1;
    slots_ = 3;
  }

  int order() const { return n_; }
  int slots() const { return slots_; }
  int products() const { return products_; }
  const std::vector<Op> &ops() const { return ops_; }

  // Step k: H <- exp(ad W_k) H cut at order n.  False when there is no odd term of order k.
  bool transform(int k) {
    auto ok = H_.find({k, 0});
    if (ok == H_.end()) return false;
    const int Ok = ok->second;
    Node w;
    w.order = k;
    w.even = false;
    w.kind = 3;
    w.src = Ok;
    const int Wk = add(w);
    gens_.push_back(Wk);
    std::map<std::pair<int, int>, std::vector<std::pair<double, int>>> parts;
    for (const auto &kv : H_) {
      const int l = kv.first.first, M = kv.second;
      parts[kv.first].push_back({1.0, M});
      int prev = M;
      double fact = 1.0;
      for (int j = 1; l + j * k <= n_; ++j) {
        fact *= j;
        Node c;
        c.order = l + j * k;
        c.even = !nodes_[prev].even;
        c.kind = 2;
        c.W = Wk;
        c.X = prev;
        const int t = add(c);
        const std::pair<int, int> key{c.order, c.even ? 1 : 0};
        parts[key].push_back({1.0 / fact, t});
        if (M == Ok) parts[key].push_back({-1.0 / (fact * (j + 1)), t});  // ad^(j+1) E0 = -ad^j O_k
        prev = t;
      }
    }
    parts[{k, 0}].clear();  // O_k + [W_k, E0] = 0
    H_.clear();
    for (auto &kv : parts) {
      auto &terms = kv.second;
      if (terms.empty()) continue;
      if (terms.size() == 1 && terms[0].first == 1.0) {
        H_[kv.first] = terms[0].second;
        continue;
      }
      Node s;
      s.order = kv.first.first;
      s.even = kv.first.second == 1;
      s.kind = 1;
      s.terms = terms;
      H_[kv.first] = add(s);
    }
    return true;
  }

  // Slots (emitting their operations) of the upper blocks of the even terms of orders 1..n
  // of the current Hamiltonian.
  std::vector<int> hamiltonian_slots() {
    std::vector<int> out;
    for (int l = 1; l <= n_; ++l) {
      auto it = H_.find({l, 1});
      if (it != H_.end()) out.push_back(slot_of(it->second, kUpper));
    }
    return out;
  }

  // (order k, slot of W_k) of every generator made so far (emitting their operations).
  std::vector<std::pair<int, int>> generator_slots() {
    std::vector<std::pair<int, int>> out;
    for (int g : gens_) out.push_back({nodes_[g].order, slot_of(g, kOdd)});
    return out;
  }

 private:
  int add(const Node &n) {
    nodes_.push_back(n);
    return (int)nodes_.size() - 1;
  }
  int fresh() { return slots_++; }

  int slot_of(int id, int part) {
    if (nodes_[id].slot[part] >= 0) return nodes_[id].slot[part];
    const Node nd = nodes_[id];  // copy: slot_of below may grow nodes_
    int d = -1;
    if (nd.kind == 3) {
      const int s = slot_of(nd.src, kOdd);
      d = fresh();
      Op op;
      op.type = kKin;
      op.dst = d;
      op.a = s;
      ops_.push_back(op);
    } else if (nd.kind == 1) {
      Op op;
      op.type = kLin;
      for (const auto &t : nd.terms) op.lin.push_back({t.first, slot_of(t.second, part)});
      d = fresh();
      op.dst = d;
      ops_.push_back(op);
    } else if (nd.kind == 2) {
      const int w = slot_of(nd.W, kOdd);
      if (nodes_[nd.X].even) {  // odd result: W X' - X W
        const int xl = slot_of(nd.X, kLower), xu = slot_of(nd.X, kUpper);
        d = fresh();
        Op g1;
        g1.type = kGemm;
        g1.dst = d;
        g1.a = w;
        g1.b = xl;
        ops_.push_back(g1);
        Op g2;
        g2.type = kGemm;
        g2.dst = d;
        g2.a = xu;
        g2.b = w;
        g2.alpha = -1.0;
        g2.beta = 1.0;
        ops_.push_back(g2);
        products_ += 2;
      } else {  // even result: one product per diagonal block
        const int xo = slot_of(nd.X, kOdd);
        const int t = fresh();
        Op g;
        g.type = kGemm;
        g.dst = t;
        g.a = w;
        g.b = xo;
        if (part == kUpper) g.adj_b = true;  // W X+
        else g.adj_a = true;                 // W+ X
        ops_.push_back(g);
        d = fresh();
        Op h;
        h.type = kHerm;
        h.dst = d;
        h.a = t;
        h.alpha = part == kUpper ? 1.0 : -1.0;
        ops_.push_back(h);
        products_ += 1;
      }
    }
    nodes_[id].slot[part] = d;
    return d;
  }

  int n_;
  int slots_ = 0;
  int products_ = 0;
  std::vector<Node> nodes_;
  std::map<std::pair<int, int>, int> H_;  // (order, even) -> node
  std::vector<int> gens_;
  std::vector<Op> ops_;
};

// Products of the DKHn Hamiltonian: the steps k <= n/2, then the final terms.
inline int hamiltonian_products(int order) {
  Plan p(order);
  for (int k = 1; k <= order / 2; ++k) p.transform(k);
  p.hamiltonian_slots();
  return p.products();
}

}  // namespace dkh
}  // namespace x2c
