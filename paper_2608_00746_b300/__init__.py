"""B300 (sm_103a) implementation of the WENO-C finite-volume operator for
compressible N-phase flows (relative-smoothness WENO weights, coupled
mass/fraction reconstruction, consistent bound-preserving limiters, HLL/HLLC
flux, SSP-RK3).  The compute path is the CUDA library ``libwenoc.so`` behind
the C ABI of ``include/wenoc.h``; ``wenoc`` is its Python binding."""
