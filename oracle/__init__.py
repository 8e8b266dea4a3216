"""FP64 CPU oracle for resonant discrete diffusion Monte Carlo (rDDMC).

TEST INFRASTRUCTURE ONLY.  Only the tests, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import anything from this package.  It
shares no code with the CUDA library in ``paper_1709_10187_gb300``; the two are
written independently from the paper (Smith et al. 2017).

Modules
-------
build     compiles ``rddmc_oracle.c`` with gcc (plain C, FP64, pthreads).
coracle   ctypes wrapper: Dawson/Voigt functions, leakage table, Philox, walks.
analytic  closed forms and exact solves used as pins: the Neufeld slab escape
          profile (Sec. 3.2, eq. Neufeld), the absorbing Markov chain of the
          DDMC walk, quadrature references for F(x), H(a,x) and bin means.
"""
