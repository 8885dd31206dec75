"""GB300-native ESP (Ewald summation with prolates) long-range electrostatics.

The solver is the CUDA library libesp_gb300.so (C-ABI in include/esp.h);
``paper_2505_09727_gb300.esp`` is its ctypes binding and
``paper_2505_09727_gb300.inputs`` builds seeded synthetic systems.
"""
