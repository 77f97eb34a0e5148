"""GB300-native MPNL uplink MIMO detection path (arXiv 2409.14355).

Submodules:
  build   -- compiles csrc/*.cu into the in-tree libmpnl.so (sm_103a)
  mpnl    -- Python binding of the C ABI in include/mpnl.h (needs a GPU)
  inputs  -- seeded synthetic slots (channel, symbols, noise); numpy only
"""
