// Generated by gen_sqrt_table.py; do not edit.
// Default six-piece rational approximant of sqrt on [0, 1]; max |error| = 9.399e-04.
#pragma once
#include "tt.cuh"
namespace spoly {
inline SqrtTable default_sqrt_table() {
  SqrtTable t;
  t.breaks[0] = 0.0;
  t.breaks[1] = 0.0004;
  t.breaks[2] = 0.007;
  t.breaks[3] = 0.048;
  t.breaks[4] = 0.2;
  t.breaks[5] = 0.65;
  t.breaks[6] = 1.0;
  t.c[0][0] = 0.000873827607193147;
  t.c[0][1] = 159.57049632636063;
  t.c[0][2] = 5957.218532826998;
  t.c[1][0] = 0.01319072330703261;
  t.c[1][1] = 22.179045003645328;
  t.c[1][2] = 147.64457357752988;
  t.c[2][0] = 0.04434930158067515;
  t.c[2][1] = 7.087002135010786;
  t.c[2][2] = 15.880992310720364;
  t.c[3][0] = 0.10329473549463793;
  t.c[3][1] = 3.12497803828535;
  t.c[3][2] = 3.1582441776128394;
  t.c[4][0] = 0.1987613970082639;
  t.c[4][1] = 1.6407938877948534;
  t.c[4][2] = 0.8787925536512886;
  t.c[5][0] = 0.29901081981926037;
  t.c[5][1] = 1.1115561191890244;
  t.c[5][2] = 0.41066562064181245;
  return t;
}
}  // namespace spoly
