// The opaque context behind the C ABI: one BlockBP problem and its engine.
#pragma once
#include "engine.h"

struct bbp_ctx {
  bbp::Engine eng;
};
