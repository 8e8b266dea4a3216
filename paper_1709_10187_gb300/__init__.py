"""GB300-native resonant discrete diffusion Monte Carlo (rDDMC) for Lyman-alpha
radiative transfer (Smith, Tsang, Bromm & Milosavljevic 2017).

The compute path is the C-ABI CUDA library built from ``csrc/`` (sm_103a);
``rddmc`` is its thin ctypes binding (argument marshalling only) and
``workloads`` describes the seeded synthetic inputs.  Importing the package does
not load the library; the first call into ``rddmc`` does, and fails loudly if it
has not been built.
"""
