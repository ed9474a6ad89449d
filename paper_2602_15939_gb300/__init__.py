"""GB300 (sm_103a) particle-in-cell step for sheared, expanding and leaky
boxes (arXiv 2602.15939).  The compute path is the CUDA library libpic
(include/pic.h); ``pic`` is its ctypes binding, ``build`` compiles it in-tree,
``workloads`` builds the seeded synthetic inputs shaped like the paper's
setups.  Importing this package loads nothing; the binding loads libpic on
first use and raises if it is missing."""
__all__ = ["pic", "build", "workloads"]
