// dna_internal.h -- declarations shared by the library's host compiler
// (dna_compile.cpp) and its CUDA side (dna_scan.cu). Not part of the public ABI.
#pragma once

#include <cstdint>
#include <string>
#include <vector>

namespace dnalib {

// Complete DFA in the dfa_load layout: table[q*4 + s], s = 0..3 for A, C, G, T;
// accept[q] = 0/1; state 0 is the start state.
struct HostDfa {
    std::vector<uint32_t> table;
    std::vector<uint8_t> accept;
    uint32_t n_states = 0;
};

// Each returns a DNA_* status code.
int compile_regex(const char *pattern, HostDfa &out);
int compile_kmers(const std::vector<std::string> &kmers, HostDfa &out);
int minimise(const HostDfa &in, HostDfa &out);

// Definite depth: the smallest m such that every word of length m sends all states
// to one state; -1 when no such m <= cap exists or when n_states > max_states (the
// analysis is quadratic in the number of states).
int definite_depth(const uint32_t *table, uint32_t n_states, int cap, uint32_t max_states);

}  // namespace dnalib
