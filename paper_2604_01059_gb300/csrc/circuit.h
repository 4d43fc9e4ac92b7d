// Stim-subset circuit representation and parser (Sec. "Methods": Tsim reads
// the Stim circuit format extended with T, T_DAG and the rotations R_X, R_Y,
// R_Z and U3, whose angles are given in units of pi).
#pragma once
#include <string>
#include <vector>

#include "common.h"

namespace tsim {

enum class Op {
  I, X, Y, Z, H, S, S_DAG, SQRT_X, SQRT_X_DAG, T, T_DAG, R_X, R_Y, R_Z, U3,
  CX, CY, CZ, SWAP,
  R, RX, M, MX, MR, MRX,
  X_ERROR, Y_ERROR, Z_ERROR, DEPOLARIZE1, PAULI_CHANNEL_1, DEPOLARIZE2, PAULI_CHANNEL_2,
  DETECTOR, OBSERVABLE_INCLUDE
};

struct Target {
  bool rec = false;  // rec[-k] target (value -k)
  int v = 0;
};

struct Instr {
  Op op;
  std::vector<double> args;
  std::vector<Target> t;
};

// One noise channel of the circuit: a group of raw error bits with a joint
// distribution (Appendix "Pauli noise channels").  Bits per qubit are (e_x,
// e_z); outcome index = sum_i bit_i << i.
struct RawChannel {
  Op kind;
  int q0 = -1, q1 = -1;
  int nbits = 0;
  std::vector<double> probs;  // size 2^nbits
  int first_bit = 0;
  int instr = 0;      // index into Circuit::ins
  int target_pos = 0; // position of (first) target within the instruction
};

struct Circuit {
  std::vector<Instr> ins;  // flattened (REPEAT unrolled), annotations kept
  int num_qubits = 0;
  int num_measurements = 0;
  std::vector<std::vector<int>> detectors;    // measurement indices
  std::vector<std::vector<int>> observables;  // measurement indices
  std::vector<RawChannel> channels;
  int num_error_bits = 0;
};

Circuit parse_circuit(const std::string& text);

}  // namespace tsim
