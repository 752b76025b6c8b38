// pdhcg_server.cu — serving loop (continuous batching); filled in below.
