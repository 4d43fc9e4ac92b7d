// Cut-order network: a message-passing graph network over the ZX diagram of a
// marginal that scores its non-Clifford spiders; the compiler cuts them in
// ascending score order.  Any cut order gives the same sum of stabilizer
// terms (Appendix "Stabilizer decompositions"), so the network only changes
// how many terms a table has, never a probability.
//
// Network (F = kCutFeatures node features, hidden width 64, three layers):
//   H0      = relu(X W_in + b_in)
//   M_l     = mean over neighbours u of H_l[u]           (0 for isolated nodes)
//   H_{l+1} = relu(H_l Ws_l + M_l Wn_l + b_l),           l = 0, 1, 2
//   s       = H3 w_o + b_o
// Weights are used in BF16; every product is accumulated in FP32.  The FP32
// master copy of the parameters has the layout
//   [W_in (F x 64, row-major) | b_in (64)]
//   3 x [Ws (64 x 64) | Wn (64 x 64) | b (64)]
//   [w_o (64) | b_o (1)]
// so that each weight matrix and its bias form one (K + 1) x J block whose
// last row is the bias.
//
// Training loss, per graph g with a set L_g of at least two labelled nodes
// (label y = log2 of the term count measured when that spider is cut first):
//   loss = (1/G) sum_g (1/|L_g|) sum_{v in L_g} ((s_v - mean_L s) - (y_v - mean_L y))^2
// with G the number of such graphs; only the order within a graph matters.
#pragma once
#include <cstdint>
#include <string>
#include <vector>

#include "common.h"

namespace tsim {
namespace cutnet {

constexpr int kHidden = 64;
constexpr int kLayers = 3;
int num_params();

// host-side graph batch: node features [n][F], CSR adjacency (symmetric,
// global node ids), graph node offsets [G + 1], labels [n] (NaN = none)
struct Batch {
  int n = 0;
  std::vector<float> X, y;
  std::vector<int> rowptr, col, goff;
};

void init_params(uint64_t seed, float* params);
// scores of every node (device execution; host buffers)
void forward(const float* params, const Batch& b, float* scores);
// loss and its gradient with respect to the BF16-rounded weights
double loss_grad(const float* params, const Batch& b, float* grad);
// Adam over minibatches of consecutive graphs; loss_per_epoch[epoch] is the
// mean minibatch loss of that epoch (before each step)
void train(const Batch& b, int epochs, int batch_graphs, float lr, uint64_t seed, float* params,
           float* loss_per_epoch);
// one Adam step of the device optimiser from given state (m, v updated in place)
void adam_step(float* params, const float* grad, float* m, float* v, int n, int step, float lr);
// registers (params != nullptr) or removes the GPU scorer used by the compiler
void set_model(const float* params);

// Held-out comparison of cut orders on graphs drawn like the training ones
// (seed, n_graphs, t_min..t_max): per graph, out[5 g ..] = non-Clifford
// spiders, terms in the heuristic order, terms with the LEARNED policy (the
// registered network; the heuristic without one), the geometric mean of the
// terms over the cut units split first (at most 16 units, the rest
// heuristic: a random first unit), and the fewest over those and the heuristic.
void evaluate_policy(uint64_t seed, int n_graphs, int t_min, int t_max, uint64_t budget, double* out);

Batch read_dataset(const std::string& path);
void write_dataset(uint64_t seed, int n_graphs, int t_min, int t_max, uint64_t budget, int max_candidates,
                   const std::string& path);

}  // namespace cutnet
}  // namespace tsim
