"""GB300 (sm_103a) silhouette-fitness library for the CMA-ES instrument tracker
of arXiv 2603.11404.

* ``workload``  seeded synthetic inputs (meshes, chain, states, masks);
* ``build``     compiles the CUDA library in-tree;
* ``api``       the C ABI's entry points on torch CUDA tensors (imported lazily:
                ``from paper_2603_11404_gb300 import api``).
"""
