/*
 * Counter-based hashing for the deterministic label propagation.
 * TEST INFRASTRUCTURE ONLY (see oracle.h).
 *
 * The paper visits vertices "in random order in parallel" (Section
 * "KaMinPar") and breaks no ties explicitly. The deterministic reading used
 * here replaces that randomness by a hash of (seed, phase tag, level, round,
 * vertex): the sub-round of vertex u is hash(u) mod S and rating ties are
 * broken by a second hash of (u, candidate).
 *
 * mix64 is the output function of splitmix64 (Steele, Lea and Flood, "Fast
 * splittable pseudorandom number generators", OOPSLA 2014), with the
 * multipliers of the public splitmix64 generator.
 */
#include "oracle.h"

#define ORC_GAMMA 0x9e3779b97f4a7c15ULL

uint64_t orc_mix64(uint64_t z) {
  z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ULL;
  z = (z ^ (z >> 27)) * 0x94d049bb133111ebULL;
  return z ^ (z >> 31);
}

/* Absorb one 64-bit word: the word is offset by the golden gamma so that a
 * zero input does not hit the fixed point mix64(0) = 0. */
uint64_t orc_step(uint64_t h, uint64_t x) { return orc_mix64(h ^ (x + ORC_GAMMA)); }

uint64_t orc_round_key(uint64_t seed, uint64_t tag, uint64_t a, uint64_t b) {
  return orc_step(orc_step(orc_step(seed, tag), a), b);
}

/* Phase tags (ASCII mnemonics packed into 64 bits). */
uint64_t orc_tag(int which) {
  switch (which) {
  case 0: return 0x4c50436c75737472ULL; /* "LPClustr": clustering LP      */
  case 1: return 0x4c50526566696e65ULL; /* "LPRefine": refinement LP      */
  case 2: return 0x54776f486f704d74ULL; /* "TwoHopMt": two-hop favourites */
  case 3: return 0x495053656564566bULL; /* "IPSeedVk": bisection seeds    */
  case 4: return 0x49504c5032576179ULL; /* "IPLP2Way": bisection LP       */
  case 5: return 0x5469654272656b72ULL; /* "TieBrekr": rating ties        */
  default: return 0;
  }
}
