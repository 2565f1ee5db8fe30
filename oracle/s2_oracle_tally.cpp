// Counting build of the oracle for its operation tally.  TEST
// INFRASTRUCTURE ONLY: compiled by oracle/tally.py, never by the product
// library.  The oracle's own source is included unchanged, with every
// double replaced by the counting type of count_double.hpp.
#include "count_double.hpp"

extern "C" {
long long or_tally[tally::SECTIONS][tally::KINDS];
int or_tally_section;

#include "s2_oracle.c"

// Zero the counters; operations outside every marked section (set-up,
// metrics) are charged to SEC_OTHER.
void or_tally_reset(void) {
  memset(or_tally, 0, sizeof(or_tally));
  or_tally_section = SEC_OTHER;
}
}
