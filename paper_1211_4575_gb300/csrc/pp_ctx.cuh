// pp_ctx.cuh -- the opaque handle of include/pp.h is the context itself.
#pragma once

#include "pp_internal.cuh"

struct pp_ctx : public pp::Ctx {};
