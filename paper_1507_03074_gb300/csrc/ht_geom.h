// Host-side geometry helpers (validation, edge tables).  Internal.
#pragma once

#include <cstdint>
#include <string>

#include "ht.h"   // include/ht.h (the build adds include/ to the search path)

namespace htg {

double snap_quarter(double a);
void theta_edges(float lo, float hi, uint32_t n, float *e);
void phi_edges(float lo, float hi, uint32_t n, float *e);
bool phi_is_full_circle(float lo, float hi);
float delta(float lo, float hi, uint32_t n);
void b_thresholds(float b_min, float db, uint32_t nb, float *beta);
uint32_t max_admit(const ht_binning &b);
bool validate(const ht_binning *b, const ht_ranges *r, uint32_t threshold, std::string *why);

} // namespace htg
