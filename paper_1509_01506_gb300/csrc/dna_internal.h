// dna_internal.h -- declarations shared by the library's host compiler
// (dna_compile.cpp) and its CUDA side (dna_scan.cu). Not part of the public ABI.
#pragma once

#include <cstdint>
#include <string>
#include <vector>

namespace dnalib {

// Complete DFA in the dfa_load layout: table[q*4 + s], s = 0..3 for A, C, G, T;
// accept[q] = the set of patterns that end when a step lands in q, as a bit mask (0 or
// 1 for a single pattern); state 0 is the start state.
struct HostDfa {
    std::vector<uint32_t> table;
    std::vector<uint32_t> accept;
    uint32_t n_states = 0;
};

// Each returns a DNA_* status code.
int compile_regex(const char *pattern, HostDfa &out);
// One automaton for several patterns (at most 32): accept[q] has bit i set when pattern
// i ends at a step that lands in q. Minimisation keeps states with different masks apart.
int compile_regex_set(const std::vector<std::string> &patterns, HostDfa &out);
int compile_kmers(const std::vector<std::string> &kmers, HostDfa &out);
int minimise(const HostDfa &in, HostDfa &out);

// Definite depth: the smallest m such that every word of length m sends all states
// to one state; -1 when no such m <= cap exists or when n_states > max_states (the
// analysis is quadratic in the number of states).
int definite_depth(const uint32_t *table, uint32_t n_states, int cap, uint32_t max_states);

}  // namespace dnalib
