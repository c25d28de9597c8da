// Request loop: continuous batching of many rank-k solves on one GPU.
#pragma once

#include "engine.h"

namespace lra {

class Server {
   public:
    explicit Server(lra_ctx *ctx);
    ~Server();
};

}  // namespace lra
