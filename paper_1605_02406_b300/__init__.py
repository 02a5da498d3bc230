"""B300-native DS-PHD/MIB dynamic occupancy grid filter (Nuss et al., Sect. VI-VII).

The compute path is the CUDA library ``libdog.so`` behind the C ABI in ``include/dog.h``;
``filter.DogFilter`` is its thin Python binding.  ``scene`` holds the seeded workload
generators.  Importing the package does not load the CUDA library; creating a filter does,
and fails loudly if it is missing.
"""
